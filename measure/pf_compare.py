"""Stein-MAP-Seq against PF-MAP-Seq on the same GPU (the paper's claim that
the Stein sets need far fewer particles, Section V-A, Table Ex1).

  python -m measure.pf_compare [--runs 50] [--T 100] [--scenario A|C]
                                              [--only stein|pf] [--N n]

Scenario A: Section V-A's constants (growth model, z = x^2/20 + r), 50 runs of
100 steps. Scenario C: the range-only zero-velocity model of Section V-C
(T = 600, six blocked periods). Stein-MAP-Seq runs with SVGD step 0.005 and
100 iterations per step at N = 10, 20, 40 (C: 20, 30, 40); PF-MAP-Seq is a
bootstrap filter with stratified resampling at every step at N = 500, 1000,
2000 (C: 1000, 2000, 4000), both followed by the same forward recursion and
backtracking. One JSON line per row:
  rmse               MAP-sequence RMSE per run, averaged over the runs (first
                     coordinate in A, position in C);
  ms_per_step_single one whole-sequence call for ONE sequence divided by its
                     steps (host copies included);
  seq_steps_per_s    time steps per second over the whole batch of runs;
  paper_rmse, paper_ms  the published figures of that row (Table Ex1; Table
                     Ex3 / Ex3_2), where the paper gives one.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from paper_2312_08684_gb300 import Estimator, workloads as W

ROWS = {
    "A": [("stein", 10, 2.0462, None), ("stein", 20, 2.1447, None), ("stein", 40, 2.2761, None),
          ("pf", 500, 7.0949, None), ("pf", 1000, 7.0696, None), ("pf", 2000, 7.1363, None)],
    "C": [("stein", 20, 0.1722, 10.82), ("stein", 30, 0.1442, 13.60), ("stein", 40, 0.1369, 16.44),
          ("pf", 1000, 0.4070, 58.94), ("pf", 2000, 0.4217, 162.01), ("pf", 4000, 0.4244, 505.32)],
}


def _workload(scenario, B, T, N):
    if scenario == "A":
        return W.make_ngm1d(B=B, T=T, N=N, L=100, step=0.005, paper_constants=True)
    return W.make_range_zv(B=B, T=T, N=N)


def _rmse(scenario, path, truth):
    k = 1 if scenario == "A" else 2
    err = path[:, 1:, :k].astype(np.float64) - truth[:, 1:, :k]
    return float(np.mean(np.sqrt(np.mean(np.sum(err ** 2, axis=2), axis=1))))


def _run(est, method, y, reps):
    fn = est.run_batch if method == "stein" else est.pf_run_batch
    fn(y)                                              # warm-up
    best, out = float("inf"), None
    for _ in range(reps):
        t0 = time.perf_counter()
        out = fn(y)
        best = min(best, time.perf_counter() - t0)
    return best, out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--scenario", choices=["A", "C"], default="A")
    ap.add_argument("--runs", type=int, default=50)
    ap.add_argument("--T", type=int, default=None)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--only", choices=["stein", "pf"], default=None, help="run the rows of one method")
    ap.add_argument("--N", type=int, default=None, help="run the rows with this particle count")
    args = ap.parse_args(argv)
    T = args.T or (100 if args.scenario == "A" else 600)
    out = []
    for method, N, paper_rmse, paper_ms in ROWS[args.scenario]:
        if (args.only and method != args.only) or (args.N and N != args.N):
            continue
        wl1 = _workload(args.scenario, 1, T, N)
        with Estimator.from_workload(wl1) as est:
            t1, _ = _run(est, method, wl1.y, args.reps)
        wl = _workload(args.scenario, args.runs, T, N)
        with Estimator.from_workload(wl) as est:
            tb, (path, J) = _run(est, method, wl.y, args.reps)
        r = {"scenario": args.scenario, "method": method, "N": N, "runs": args.runs, "T": T,
             "rmse": _rmse(args.scenario, path, wl.truth), "paper_rmse": paper_rmse,
             "ms_per_step_single": 1e3 * t1 / T, "paper_ms": paper_ms,
             "seq_steps_per_s": args.runs * T / tb, "J_finite": bool(np.all(np.isfinite(J)))}
        out.append(r)
        print(json.dumps(r), flush=True)
    return out


if __name__ == "__main__":
    main()
