"""Range-only localisation without a motion prior (the paper's Section V-C form).

  python -m measure.scenario_c [--runs 64] [--T 600] [--prior 0|2]
                                             [--N n] [--variant v]

2-D position, zero-velocity random walk with Q = (alpha dt)^2 I = 0.01 I, range
measurements to three anchors with sigma_z = 0.5, anchor 1 blocked for six
periods (2.5, 5.0, 4.0, 4.0, 3.0 and 3.5 s at 10 Hz), SVGD step 0.005 and 100
iterations per step, median bandwidth, and the transition-mixture prior
(--prior 0) or the prior conditioned on the previous MAP estimates that the
section describes (--prior 2: the best predecessor under phi_{t-1}). The
trajectories are seeded synthetic random walks (the paper's recorded
trajectories are not available), so the RMSE column is compared in
magnitude only.

Per particle count (Table Ex3 / Table Ex3_2 rows N = 20, 30, 40) it prints one
JSON line with
  - ms_per_step_single: wall time of one whole-sequence call for ONE sequence
    (host copies included) divided by its time steps: the latency a single
    online estimator sees per measurement, against the paper's per-step time;
  - seq_steps_per_s_batched: time steps per second with --runs sequences in
    one batched call (the data-parallel throughput);
  - rmse: position RMSE of the MAP sequence per run, averaged over the runs.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from paper_2312_08684_gb300 import Estimator, workloads as W

# N -> (the paper's Stein-MAP-Seq RMSE in m, its computation time in ms)
PAPER = {20: (0.1722, 10.82), 30: (0.1442, 13.60), 40: (0.1369, 16.44)}


def rmse_of(path, truth):
    err = path[:, 1:, :2].astype(np.float64) - truth[:, 1:, :2]
    return float(np.mean(np.sqrt(np.mean(np.sum(err ** 2, axis=2), axis=1))))


def _timed(est, y, reps, variant=None):
    if variant is not None:
        est.set_variant(variant)
    est.run_batch(y)                                   # warm-up (graph capture, first launch)
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        path, J = est.run_batch(y)
        best = min(best, time.perf_counter() - t0)
    return best, path, J


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs", type=int, default=64)
    ap.add_argument("--T", type=int, default=600)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--prior", type=int, default=W.PRIOR_MIXTURE, choices=[0, 1, 2])
    ap.add_argument("--N", type=int, default=None, help="run only this particle count")
    ap.add_argument("--variant", type=int, default=None,
                    help="step-kernel variant (smap_set_variant; default: the built-in choice)")
    args = ap.parse_args(argv)
    out = []
    for N, (paper_rmse, paper_ms) in PAPER.items():
        if args.N and N != args.N:
            continue
        wl1 = W.make_range_zv(B=1, T=args.T, N=N, prior=args.prior)
        with Estimator.from_workload(wl1) as est:
            t1, _, _ = _timed(est, wl1.y, args.reps, args.variant)
            variant = est.variant()
        wl = W.make_range_zv(B=args.runs, T=args.T, N=N, prior=args.prior)
        with Estimator.from_workload(wl) as est:
            tb, path, J = _timed(est, wl.y, args.reps, args.variant)
        r = {"N": N, "L": wl.L, "T": args.T, "runs": args.runs, "prior": args.prior,
             "variant_single": list(variant),
             "ms_per_step_single": 1e3 * t1 / args.T, "paper_ms_per_step": paper_ms,
             "seq_steps_per_s_batched": args.runs * args.T / tb,
             "rmse": rmse_of(path, wl.truth), "paper_rmse": paper_rmse,
             "J_finite": bool(np.all(np.isfinite(J)))}
        out.append(r)
        print(json.dumps(r), flush=True)
    return out


if __name__ == "__main__":
    main()
