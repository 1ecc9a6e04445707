"""Writes tests/golden/cfg1_oracle_snapshot.txt by calling only the oracle.

The snapshot is a regression record of the FP64 oracle on the 256x256, 10k-Gaussian
scene (Eq. 1-4 under Algorithm 5's rules): any later change to the oracle's arithmetic
shows up as a diff of this file, and the commit that changes it must name the passage
of the paper that justifies the change.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2412_17378_gb300 import scenes  # noqa: E402

PIXELS = [0, 777, 12345, 32896, 40000, 65535]


def snapshot():
    s = scenes.scene_config("cfg1")
    g, cam = s["gaussians"], s["cameras"][0]
    pp = oracle.preprocess(g["means3D"], g["log_scales"], g["quats"], g["opacities"], cam)
    m2, co, dp = (pp[k].astype(np.float32) for k in ("means2D", "conic_opacity", "depth"))
    pl, rg = oracle.bin_tiles(m2, pp["radius"], dp, 256, 256)
    out = oracle.render(m2, co, g["colors"], dp, pl, rg, 256, 256)
    rows = [("K", int(pl.size)), ("sum_n_eval", int(out["n_eval"].sum())),
            ("sum_n_contrib", int(out["n_contrib"].sum())), ("sum_n_acc", int(out["n_acc"].sum()))]
    for p in PIXELS:
        rows.append((f"color_r_{p}", float(out["color"][0].ravel()[p])))
        rows.append((f"final_T_{p}", float(out["final_T"].ravel()[p])))
    return rows


if __name__ == "__main__":
    with open(os.path.join(HERE, "cfg1_oracle_snapshot.txt"), "w") as f:
        f.write("# FP64 oracle on the 256x256 / 10k-Gaussian scene (seed 0); Eq. 4 + Algorithm 5.\n")
        f.write("# written by tests/golden/make_golden.py (oracle only)\n")
        for k, v in snapshot():
            f.write(f"{k} {v!r}\n")
