"""The forward recursion alone (smap_viterbi) on particle sets from a real run.

  python -m measure.recursion [--config C2|C3|C4] [--B 1024] [--reps 3] [--variant V]

Runs the configuration's batched method once (the particle sets SVGD
produces), then times smap_viterbi on those sets with CUDA events on the
handle's stream and prints one JSON line: milliseconds per run, the
recursion's algorithmic operations (2d+2 per ordered pair of consecutive
particle sets) against the FP32 issue peak, and the recursion counters
(particle-steps, near-ties, exact candidate scores). Used for the recursion's
ncu captures (profiles/recursion_*.md).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2312_08684_gb300 import Estimator, _binding as abi  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="C3", choices=["C2", "C3", "C4"])
    ap.add_argument("--B", type=int, default=1024)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--variant", type=int, default=None, help="launch shape of the recursion (smap_set_variant)")
    args = ap.parse_args(argv)
    import torch
    wl = bench.make_workload(args.config, 0, args.B)
    stream = torch.cuda.Stream()
    y = torch.from_numpy(wl.y).cuda()
    path = torch.empty((wl.B, wl.maxT + 1, wl.d), dtype=torch.float32, device="cuda")
    J = torch.empty(wl.B, dtype=torch.float64, device="cuda")
    T = np.ascontiguousarray(wl.T, np.int32)
    with Estimator.from_workload(wl, stream=stream) as est:
        abi.smap_run_batch(est.h, y, T, None, path, J)
        batch_ms = abi.smap_last_kernel_ms(est.h)[0]
        hist = torch.empty((wl.B, wl.maxT, wl.N, wl.d), dtype=torch.float32, device="cuda")
        abi.smap_get_history(est.h, hist)
        abi.smap_debug_recursion_stats(est.h)
        if args.variant is not None:
            est.set_variant(args.variant)
        ms = []
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                e0.record(stream)
                abi.smap_viterbi(est.h, hist, y, T, None, path, J)
                e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        n_ps, n_tie, n_eval = abi.smap_debug_recursion_stats(est.h)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    pk, _ = bench.peaks()
    peak = bench.alu_peak_gops(pk.get("sm_max_mhz", 2070.0), sms)
    ops = bench.recursion_ops(wl)
    best = min(ms)
    print(json.dumps({"config": args.config, "B": wl.B, "N": wl.N, "d": wl.d, "variant": args.variant,
                      "batch_kernel_ms": batch_ms,
                      "viterbi_ms": ms, "achieved_gops": ops / (best / 1e3) / 1e9, "peak_gops": peak,
                      "frac": ops / (best / 1e3) / 1e9 / peak, "particle_steps": n_ps,
                      "near_tie_fraction": n_tie / max(n_ps, 1),
                      "exact_scores_per_particle_step": n_eval / max(n_ps, 1)}), flush=True)


if __name__ == "__main__":
    main()
