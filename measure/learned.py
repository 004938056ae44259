"""Learned-proposal benchmark: plain SVGD with L iterations per step against
the learned initialisation with a few iterations, on the same GB300.

  python -m measure.learned --workload arm|clutter [options]
  python -m measure.learned --forward-only ROWS [--reps K]

1. Training data: plain runs (L_plain iterations) of sequences disjoint from
   the evaluation set; smap_proposal_capture turns every (sequence, step,
   particle) into a row (features of the plain initialisation, displacement
   to the final particle).
2. Training: smap_proposal_train (the library's forward/backward/Adam
   kernels) on minibatches of those rows. With --rounds R > 1, each further
   round regenerates the training runs with L_plain iterations started from
   the previous round's network and trains a fresh network on them
   (self-distillation: the targets are particles after more SVGD progress).
3. Evaluation on fresh sequences: device time of smap_run_batch (resident
   observations, CUDA events inside the run's graph) and the mean MAP
   log-posterior J for plain L_plain, plain L_learned and learned L_learned.
Prints one JSON line. All arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from paper_2312_08684_gb300 import Estimator, _binding as abi, workloads as W


def _make(which, B, T, N, L, first, seed):
    """Workload of the arm (fixed T) or clutter shape; clutter with T=None has
    the batched configuration's uneven lengths, T ~ U[50, 400]."""
    if which == "arm":
        return W.make_planar_arm(B=B, T=T, N=N, L=L, first=first, seed=seed)
    if T is None:
        return W.make_clutter_cv(B=B, N=N, L=L, first=first, seed=seed)
    return W.make_clutter_cv(B=B, Tmin=T, Tmax=T, N=N, L=L, first=first, seed=seed)


def _run(torch, wl, L, prop=None, reps=1):
    """Batched run of wl with L SVGD iterations per step (and the proposal, if
    given). The time of a run is its device time from the CUDA events the
    library records inside the batched run's graph (state reset to the end of
    backtracking; observations resident on the device), so recording the graph
    on the first run does not count. Returns the median seconds and J."""
    stream = torch.cuda.Stream()
    with Estimator.from_workload(wl, L=L, stream=stream) as est:
        if prop is not None:
            abi.smap_set_proposal(est.h, prop, L)
        y = torch.from_numpy(wl.y).cuda()
        path = torch.empty((wl.B, wl.maxT + 1, wl.d), dtype=torch.float32, device="cuda")
        J = torch.empty(wl.B, dtype=torch.float64, device="cuda")
        T = np.ascontiguousarray(wl.T, np.int32)
        times = []
        for _ in range(reps):
            abi.smap_run_batch(est.h, y, T, None, path, J)
            times.append(abi.smap_last_kernel_ms(est.h)[1] / 1000.0)
        Jh = J.cpu().numpy()
    if not np.all(np.isfinite(Jh)):
        raise RuntimeError("non-finite MAP score")
    return float(np.median(times)), Jh


def compare(which, N=None, T=100, train_seqs=1000, eval_seqs=4096, L_plain=50, L_learned=5, steps=4000,
            batch=8192, lr=1e-3, max_rows=1.2e8, rounds=3, reps=1, log=None):
    """Learned L_learned vs plain L_plain on eval_seqs fresh sequences.

    Round 1 trains on rows captured from plain runs (L_plain iterations from
    the plain initialisation) of train_seqs sequences disjoint from the
    evaluation set; each further round regenerates the rows with runs started
    from the previous round's network (self-distillation) and trains a fresh
    network. The learned form is evaluated after every round; speed and mean J
    of plain L_plain and plain L_learned are measured once."""
    import torch
    N = N or (1024 if which == "arm" else 512)
    probe = _make(which, 1, 2, N, L_plain, 0, 100)
    ev = _make(which, eval_seqs, T, N, L_learned, 0, 4)
    mean_T = float(np.mean(ev.T))
    total = min(int(max_rows), int(train_seqs * mean_T * 1.5) * N)
    feat = torch.empty((total, abi.MLP_IN_P), dtype=torch.float32, device="cuda")
    targ = torch.empty((total, abi.MLP_OUT_P), dtype=torch.float32, device="cuda")
    prop, history = None, []
    for rnd in range(rounds):
        nxt = abi.smap_proposal_create(probe.kind, probe.params, seed=7 + rnd)
        rows, done, steps_seen, chunk = 0, 0, 0, 304
        t0 = time.time()
        while done < train_seqs and rows < total:
            b = min(chunk, train_seqs - done)
            wl = _make(which, b, T, N, L_plain, 100000 + done, 100)
            if rows + int(np.sum(wl.T)) * N > total:
                break
            with Estimator.from_workload(wl) as est:
                if prop is not None:
                    abi.smap_set_proposal(est.h, prop, L_plain)
                est.run_batch(wl.y, wl.T)
                rows += abi.smap_proposal_capture(nxt, est.h, feat[rows:], targ[rows:])
            done += b
            steps_seen += int(np.sum(wl.T))
        t_data = time.time() - t0
        abi.smap_proposal_fit_normalization(nxt, feat[:rows], targ[:rows])
        t1 = time.time()
        curve = abi.smap_proposal_train(nxt, feat[:rows], targ[:rows], steps, batch, lr, lr * 0.05)
        torch.cuda.synchronize()
        t_train = time.time() - t1
        if prop is not None:
            abi.smap_proposal_destroy(prop)
        prop = nxt
        t_l, J_l = _run(torch, ev, L_learned, prop, reps=reps if rnd == rounds - 1 else 1)
        history.append({"round": rnd + 1, "data": "plain runs" if rnd == 0 else "runs from the previous network",
                        "rows": rows, "sequence_steps": steps_seen, "adam_steps": steps, "batch": batch,
                        "loss_first": float(np.mean(curve[:20])), "loss_last": float(np.mean(curve[-50:])),
                        "data_seconds": t_data, "train_seconds": t_train,
                        "learned_seconds": t_l, "learned_mean_J": float(np.mean(J_l))})
        if log:
            log(history[-1])
    del feat, targ
    torch.cuda.empty_cache()
    abi.smap_proposal_destroy(prop)
    t_plain, J_plain = _run(torch, ev, L_plain, reps=reps)
    t_small, J_small = _run(torch, ev, L_learned, reps=reps)
    mp, ms = float(np.mean(J_plain)), float(np.mean(J_small))
    t_learn = history[-1]["learned_seconds"]

    def gap(mj):
        return (mp - mj) / abs(mp)

    Tdesc = f"T={T}" if T is not None else f"T~U[{int(ev.T.min())},{int(ev.T.max())}]"
    return {
        "workload": f"{which}: N={N}, {Tdesc}, d={ev.d}, {eval_seqs} evaluation sequences",
        "plain": {"L": L_plain, "seconds": t_plain, "sequences_per_s": ev.B / t_plain, "mean_J": mp},
        "plain_small_L": {"L": L_learned, "seconds": t_small, "sequences_per_s": ev.B / t_small, "mean_J": ms},
        "learned": {"L": L_learned, "seconds": t_learn, "sequences_per_s": ev.B / t_learn,
                    "mean_J": history[-1]["learned_mean_J"]},
        "speedup_learned_vs_plain": t_plain / t_learn,
        "J_gap_rel_plain_data": gap(history[0]["learned_mean_J"]),
        "J_gap_rel": gap(history[-1]["learned_mean_J"]),
        "J_gap_rel_without_network": gap(ms),
        "timing": "device time of each batched run (CUDA events inside its graph), observations resident",
        "training": history,
    }


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
    ap.add_argument("--T", type=int, default=100, help="steps per sequence (clutter: 0 = U[50, 400])")
    ap.add_argument("--train-seqs", type=int, default=1000, help="training sequences per round")
    ap.add_argument("--eval-seqs", type=int, default=4096)
    ap.add_argument("--L-plain", type=int, default=50)
    ap.add_argument("--L-learned", type=int, default=5)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--max-rows", type=float, default=1.2e8)
    ap.add_argument("--rounds", type=int, default=3, help="self-distillation rounds (1 = plain-run data only)")
    ap.add_argument("--reps", type=int, default=1, help="timed repetitions of each evaluation run (median)")
    ap.add_argument("--forward-only", type=int, default=0, metavar="ROWS",
                    help="only time the network's inference forward on ROWS rows")
    args = ap.parse_args(argv)
    if args.forward_only:
        return forward_only(args.forward_only, max(args.reps, 1))
    out = compare(args.workload, N=args.N, T=args.T or None, train_seqs=args.train_seqs,
                  eval_seqs=args.eval_seqs, L_plain=args.L_plain, L_learned=args.L_learned, steps=args.steps,
                  batch=args.batch, lr=args.lr, max_rows=args.max_rows, rounds=args.rounds, reps=args.reps)
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
