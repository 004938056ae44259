"""Learned-proposal benchmark: plain SVGD with L iterations per step against
the learned initialisation with a few iterations, on the same GB300.

  python -m paper_2312_08684_gb300.learned --workload arm|clutter [options]
  python -m paper_2312_08684_gb300.learned --forward-only ROWS [--reps K]

1. Training data: plain runs (L_plain iterations) of sequences disjoint from
   the evaluation set; smap_proposal_capture turns every (sequence, step,
   particle) into a row (features of the plain initialisation, displacement
   to the final particle).
2. Training: smap_proposal_train (the library's forward/backward/Adam
   kernels) on minibatches of those rows. With --rounds R > 1, each further
   round regenerates the training runs with L_plain iterations started from
   the previous round's network and trains a fresh network on them
   (self-distillation: the targets are particles after more SVGD progress).
3. Evaluation on fresh sequences: wall time of smap_run_batch (device-resident
   observations, CUDA events) and the mean MAP log-posterior J for plain
   L_plain, plain L_learned and learned L_learned.
Prints one JSON line. All arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import Estimator, _binding as abi, workloads as W


def _make(which, B, T, N, L, first, seed):
    if which == "arm":
        return W.make_planar_arm(B=B, T=T, N=N, L=L, first=first, seed=seed)
    return W.make_clutter_cv(B=B, Tmin=T, Tmax=T, N=N, L=L, first=first, seed=seed)


def _run(torch, wl, L, prop=None, reps=2):
    stream = torch.cuda.Stream()
    with Estimator.from_workload(wl, L=L, stream=stream) as est:
        if prop is not None:
            abi.smap_set_proposal(est.h, prop, L)
        y = torch.from_numpy(wl.y).cuda()
        path = torch.empty((wl.B, wl.maxT + 1, wl.d), dtype=torch.float32, device="cuda")
        J = torch.empty(wl.B, dtype=torch.float64, device="cuda")
        T = np.ascontiguousarray(wl.T, np.int32)
        abi.smap_run_batch(est.h, y, T, None, path, J)      # records the graph
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                abi.smap_run_batch(est.h, y, T, None, path, J)
                e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1000.0)
        Jh = J.cpu().numpy()
    if not np.all(np.isfinite(Jh)):
        raise RuntimeError("non-finite MAP score")
    return float(np.min(times)), Jh


def forward_only(rows, reps):
    """Times the inference forward (the tensor-core kernel) alone on `rows`
    random standardised feature rows of the clutter network shape."""
    import torch
    probe = _make("clutter", 1, 2, 512, 5, 0, 100)
    p = abi.smap_proposal_create(probe.kind, probe.params, seed=3)
    n_in, n_out, _, _ = abi.smap_proposal_dims(p)
    g = torch.Generator(device="cuda").manual_seed(1)
    feat = torch.zeros((rows, abi.MLP_IN_P), dtype=torch.float32, device="cuda")
    feat[:, :n_in] = torch.randn((rows, n_in), device="cuda", generator=g)
    disp = torch.empty((rows, n_out), dtype=torch.float32, device="cuda")
    for _ in range(3):
        abi.smap_proposal_forward(p, feat, disp)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        abi.smap_proposal_forward(p, feat, disp)   # synchronous
        ts.append(time.perf_counter() - t0)
    abi.smap_proposal_destroy(p)
    t = float(np.median(ts))
    flop = 2.0 * rows * (abi.MLP_IN_P * abi.MLP_H + abi.MLP_H * abi.MLP_H + abi.MLP_H * abi.MLP_OUT_P)
    out = {"forward_rows": rows, "ms": t * 1e3, "tflops_padded": flop / t / 1e12,
           "timing": "host wall clock around the synchronous call, median of reps",
           "finite": bool(torch.isfinite(disp).all())}
    print(json.dumps(out), flush=True)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="arm", choices=["arm", "clutter"])
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--T", type=int, default=100)
    ap.add_argument("--train-seqs", type=int, default=1000, help="training sequences (x T steps)")
    ap.add_argument("--eval-seqs", type=int, default=4096)
    ap.add_argument("--L-plain", type=int, default=50)
    ap.add_argument("--L-learned", type=int, default=5)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--max-rows", type=float, default=1.2e8)
    ap.add_argument("--rounds", type=int, default=3, help="self-distillation rounds (1 = plain-run data only)")
    ap.add_argument("--reps", type=int, default=1, help="timed repetitions of each evaluation run")
    ap.add_argument("--forward-only", type=int, default=0, metavar="ROWS",
                    help="only time the network's inference forward on ROWS rows")
    args = ap.parse_args(argv)
    if args.forward_only:
        return forward_only(args.forward_only, max(args.reps, 1))
    import torch
    which = args.workload
    N = args.N or (1024 if which == "arm" else 512)
    t0 = time.time()
    probe = _make(which, 1, 2, N, args.L_plain, 0, 100)
    total = min(int(args.max_rows), args.train_seqs * args.T * N)
    feat = torch.empty((total, abi.MLP_IN_P), dtype=torch.float32, device="cuda")
    targ = torch.empty((total, abi.MLP_OUT_P), dtype=torch.float32, device="cuda")
    ev = _make(which, args.eval_seqs, args.T, N, args.L_learned, 0, 4)
    prop, history = None, []
    for rnd in range(args.rounds):
        # 1. training data from runs with L_plain iterations (chunks of sequences);
        #    from the second round on, started from the previous network
        nxt = abi.smap_proposal_create(probe.kind, probe.params, seed=7 + rnd)
        rows, done, chunk = 0, 0, 304
        t0 = time.time()
        while done < args.train_seqs and rows < total:
            b = min(chunk, args.train_seqs - done)
            wl = _make(which, b, args.T, N, args.L_plain, 100000 + done, 100)
            with Estimator.from_workload(wl) as est:
                if prop is not None:
                    abi.smap_set_proposal(est.h, prop, args.L_plain)
                est.run_batch(wl.y, wl.T)
                need = wl.B * wl.maxT * N
                if rows + need > total:
                    break
                rows += abi.smap_proposal_capture(nxt, est.h, feat[rows:], targ[rows:])
            done += b
        t_data = time.time() - t0
        # 2. training
        abi.smap_proposal_fit_normalization(nxt, feat[:rows], targ[:rows])
        t1 = time.time()
        curve = abi.smap_proposal_train(nxt, feat[:rows], targ[:rows], args.steps, args.batch, args.lr,
                                        args.lr * 0.05)
        torch.cuda.synchronize()
        t_train = time.time() - t1
        if prop is not None:
            abi.smap_proposal_destroy(prop)
        prop = nxt
        history.append({"rows": rows, "sequence_steps": done * args.T, "steps": args.steps, "batch": args.batch,
                        "loss_first": float(np.mean(curve[:20])), "loss_last": float(np.mean(curve[-50:])),
                        "data_seconds": t_data, "train_seconds": t_train})
        if args.rounds > 1:
            history[-1]["learned_mean_J"] = float(np.mean(_run(torch, ev, args.L_learned, prop, reps=1)[1]))
    del feat, targ
    torch.cuda.empty_cache()
    # 3. evaluation on fresh sequences
    t_plain, J_plain = _run(torch, ev, args.L_plain, reps=args.reps)
    t_small, J_small = _run(torch, ev, args.L_learned, reps=args.reps)
    t_learn, J_learn = _run(torch, ev, args.L_learned, prop, reps=args.reps)
    abi.smap_proposal_destroy(prop)
    mp, ml, ms = float(np.mean(J_plain)), float(np.mean(J_learn)), float(np.mean(J_small))
    out = {
        "workload": f"{which}: N={N}, T={args.T}, d={ev.d}, {args.eval_seqs} evaluation sequences",
        "plain": {"L": args.L_plain, "seconds": t_plain, "sequences_per_s": ev.B / t_plain, "mean_J": mp},
        "plain_small_L": {"L": args.L_learned, "seconds": t_small, "sequences_per_s": ev.B / t_small,
                          "mean_J": ms},
        "learned": {"L": args.L_learned, "seconds": t_learn, "sequences_per_s": ev.B / t_learn, "mean_J": ml},
        "speedup_learned_vs_plain": t_plain / t_learn,
        "J_gap_rel": (mp - ml) / abs(mp),
        "J_gap_rel_without_network": (mp - ms) / abs(mp),
        "training": history,
    }
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
