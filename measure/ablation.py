"""Kernel / bandwidth / particle-count ablation on the paper's scenario A.

  python -m measure.ablation [--runs 50] [--T 100]

Scenario A with the constants of Section V-A (growth model, z = x^2/20 + r,
v ~ N(0,5), r ~ N(0,16), x_0 ~ N(0,5)), SVGD step 0.005, 100 iterations per
step, median-heuristic bandwidth h (times the scale of the row), as in the
paper's kernel ablation (Table Ex6). Each row: MAP-sequence RMSE per run,
averaged over the runs, computed on the GPU (the batch is the Monte Carlo
runs). Prints one JSON line per row with the paper's published value beside
it (the paper's random draws and initialisation are not reproducible, so the
comparison is of magnitude and trends, not of values).
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from paper_2312_08684_gb300 import Estimator, workloads as W

# (kernel, bandwidth scale, N) -> the paper's RMSE (Table Ex6)
ROWS = [
    ("RBF", 1.0, 10, 2.2643), ("IMQ", 1.0, 10, 2.2512), ("Matern", 1.0, 10, 2.2344),
    ("RBF", 0.5, 10, 2.4887), ("RBF", 3.0, 10, 2.0462), ("RBF", 0.5, 40, 2.2507), ("RBF", 3.0, 40, 2.1970),
    ("RBF", 1.0, 20, 2.2108), ("RBF", 1.0, 40, 2.1369), ("IMQ", 1.0, 20, 2.1557), ("IMQ", 1.0, 40, 2.1780),
    ("Matern", 1.0, 20, 2.1232), ("Matern", 1.0, 40, 2.0714),
]
KERNEL = {"RBF": 0, "IMQ": 1, "Matern": 2}


def rmse_of(path, truth):
    err = path[:, 1:, 0].astype(np.float64) - truth[:, 1:, 0]
    return float(np.mean(np.sqrt(np.mean(err ** 2, axis=1))))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs", type=int, default=50)
    ap.add_argument("--T", type=int, default=100)
    args = ap.parse_args(argv)
    out = []
    for kern, scale, N, paper in ROWS:
        wl = W.make_ngm1d(B=args.runs, T=args.T, N=N, L=100, step=0.005, paper_constants=True,
                          bw_value=scale)
        wl.kernel = KERNEL[kern]
        with Estimator.from_workload(wl) as est:
            path, J = est.run_batch(wl.y)
        r = {"kernel": kern, "bandwidth_scale": scale, "N": N, "rmse": rmse_of(path, wl.truth),
             "paper_rmse": paper, "runs": args.runs, "T": args.T}
        out.append(r)
        print(json.dumps(r), flush=True)
    return out


if __name__ == "__main__":
    main()
