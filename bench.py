"""Benchmark of the Stein-MAP-Seq hot path on GB300.

One "step" = one whole batched run of the workload through the C ABI
(smap_run_batch). The default workload is the data-association one: 4096
sequences of a 2-D constant-velocity target (d=4) observed through 10 points
per step (one true, the rest clutter, 20% of steps without the true point),
lengths T ~ U[50, 400], N=512 particles, L=30 SVGD iterations per time step,
followed by the Viterbi recursion and backtracking. Metric: SVGD
particle-updates/s (sum over sequences of N L T divided by the step time) and
sequences/s. After the timed steps the same process times the learned
proposal (L=5 SVGD iterations from the network's initialisation) against
plain SVGD with L=50 on the data-association shape and on the 7-link arm
shape (4096 sequences each), with the networks trained on the GPU first.

  python bench.py [--gpus N --steps K --warmup W] [--impl smap|reference]
                  [--config C1|C2|C3|C4] [--no-c5] [--no-autotune]

Under torchrun (N > 1) each rank runs its own sequences (weak scaling, no
collective on the data path); rank 0 prints the JSON line with the time maxed
over ranks. --impl reference times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2312_08684_gb300 import workloads as W  # noqa: E402

METRIC = "SVGD particle-updates/s"
UNIT = "particle-updates/s"
CSRC = os.path.join(ROOT, "paper_2312_08684_gb300", "csrc")

# name: (builder(B, first), description, oracle sample steps, instantiation unit)
CONFIGS = {
    "C1": (lambda B, first: W.make_ngm1d(),
           "ngm1d: 1-D growth model, sign-ambiguous z = x^2/20, N=32, L=50, T=50, one sequence", 50,
           "smap_inst_ngm1d.cu"),
    "C2": (lambda B, first: W.make_range_cv(B=B, first=first),
           "range_cv: 2-D range-only CV (d=4, 3 beacons, beacons 2-3 silent for steps 60-120), "
           "N=256, L=30, T=200", 30, "smap_inst_range_cv.cu"),
    "C3": (lambda B, first: W.make_clutter_cv(B=B, first=first),
           "clutter_cv: 2-D CV target (d=4) in clutter, 10 points per step (1 true, 20% of steps "
           "none), unknown association with an outlier term, N=512, L=30, T~U[50,400]", 30,
           "smap_inst_clutter_cv.cu"),
    "C4": (lambda B, first: W.make_planar_arm(B=B, first=first),
           "planar_arm: 7-link planar chain (d=14), end-effector observation, N=1024, L=50, T=100", 2,
           "smap_inst_planar_arm7.cu"),
}
DEFAULT_CONFIG = "C3"
DEFAULT_B = {"C1": 1, "C2": 1024, "C3": 4096, "C4": 256}


def shard(rank: int, world: int, B: int):
    """Sequence ids of one rank under weak scaling: rank r owns [r B, (r+1) B)."""
    return list(range(rank * B, (rank + 1) * B))


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The slowest rank's time (the job's time under weak scaling)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_workload(config: str, rank: int, B: int | None = None):
    """The configuration's workload for one rank: B sequences (default: the
    configuration's batch) numbered from rank * B."""
    B = B or DEFAULT_B[config]
    return CONFIGS[config][0](B, rank * B)


def algorithmic_ops(wl) -> float:
    """FP32/SFU lane operations the method needs (per ordered pair-iteration
    8d+8: RBF kernel and update 4d+1 + exp, mixture prior 3d+4 + exp, median
    d+1; per ordered pair-step of the recursion 2d+2: d differences, d
    weighted squares, one add of the previous score, one comparison)."""
    d = wl.d
    n2 = wl.Nseq.astype(np.float64) ** 2
    T = wl.T.astype(np.float64)
    return float(np.sum(n2 * T * (wl.L * (8 * d + 8) + (2 * d + 2))))


def recursion_ops(wl) -> float:
    """Lane operations of the Viterbi recursion alone (2d+2 per ordered pair
    of consecutive particle sets; the first step has one predecessor)."""
    d = wl.d
    n = wl.Nseq.astype(np.float64)
    T = wl.T.astype(np.float64)
    return float(np.sum((n * n * (T - 1) + n) * (2 * d + 2)))


def kernel_source_sha(config: str) -> str:
    """Digest of the sources the step kernel of this configuration compiles
    from; a traffic figure taken on other sources no longer applies."""
    h = hashlib.sha256()
    for name in ("smap_kernels.cuh", "smap_models.cuh", "smap_common.cuh", "smap_internal.h",
                 CONFIGS[config][3]):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def seq_kernel_traffic(config: str, wl):
    """DRAM bytes (read + write) of one step-kernel launch on this workload,
    from the committed ncu summary of the same configuration and kernel
    sources (profiles/seq_kernel_<workload>_traffic.md); None when there is
    none for this configuration, size and source digest."""
    path = os.path.join(ROOT, "profiles", f"seq_kernel_{wl.name}_traffic.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if line.startswith("traffic:"):
                for kv in line[len("traffic:"):].split():
                    k, v = kv.split("=")
                    vals[k] = v
    want = {"B": str(wl.B), "N": str(wl.N), "L": str(wl.L), "T": str(int(wl.T.sum())),
            "source": kernel_source_sha(config)}
    if any(vals.get(k) != v for k, v in want.items()):
        return None
    return int(vals["bytes_per_launch"])


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def alu_peak_gops(sm_mhz: float, sms: int) -> float:
    """FP32 issue peak: 128 lanes per SM per clock (4 sub-partitions x 32)."""
    return sms * 128 * sm_mhz * 1e6 / 1e9


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(wl_full, threads: int, T_sample: int):
    """The FP64 oracle as it stands, one sequence per host thread, T_sample steps."""
    from oracle import oracle as O
    O.lib()
    nseq = min(threads, wl_full.B)
    sub = wl_full.subset(np.arange(nseq))
    T_sample = min(T_sample, int(sub.T.min()))
    T = np.full(nseq, T_sample, np.int32)
    t0 = time.perf_counter()
    O.run_batch(sub.kind, sub.params, sub.N, sub.L, sub.step, sub.bw_rule, sub.bw_value, sub.prior,
                sub.seed, np.arange(nseq), sub.x0, sub.y[:, :T_sample].astype(np.float64), T,
                nthreads=threads)
    dt = time.perf_counter() - t0
    units = nseq * sub.N * sub.L * T_sample
    return {"value": units / dt, "unit": UNIT, "cores": nseq, "kind": "oracle",
            "sample": f"{nseq} sequences x first {T_sample} steps (N={sub.N}, L={sub.L}), one sequence "
                      f"per host thread, {dt:.1f} s"}


def all_configs(args):
    """One JSON line per configuration (one GPU): batched run of the whole
    configuration timed with CUDA events (inputs resident), the step kernel's
    ALU roofline, the recursion alone, and the oracle on a bounded sample."""
    import torch
    from paper_2312_08684_gb300 import Estimator, _binding as abi
    pk, src = peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = alu_peak_gops(pk.get("sm_max_mhz", 2070.0), sms)
    abi_grid = {}
    for name, (mk, desc, t_sample, _) in CONFIGS.items():
        wl = make_workload(name, 0)
        stream = torch.cuda.Stream()
        y = torch.from_numpy(wl.y).cuda()
        path = torch.empty((wl.B, wl.maxT + 1, wl.d), dtype=torch.float32, device="cuda")
        J = torch.empty(wl.B, dtype=torch.float64, device="cuda")
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Estimator.from_workload(wl, stream=stream) as est:
            def timed(fn, reps):
                ms = []
                for _ in range(reps):
                    torch.cuda.synchronize()
                    with torch.cuda.stream(stream):
                        ev0.record(stream)
                        fn()
                        ev1.record(stream)
                    ev1.synchronize()
                    ms.append(ev0.elapsed_time(ev1))
                return float(np.mean(ms))
            run = lambda: abi.smap_run_batch(est.h, y, wl.T, wl.Nseq, path, J)
            for _ in range(max(args.warmup, 3)):
                run()
            ms = timed(run, args.steps)
            kms = abi.smap_last_kernel_ms(est.h)[0]
            abi_grid[name] = abi.smap_get_variant(est.h)
            hist = torch.empty((wl.B, wl.maxT, wl.N, wl.d), dtype=torch.float32, device="cuda")
            abi.smap_get_history(est.h, hist)
            vit = lambda: abi.smap_viterbi(est.h, hist, y, wl.T, wl.Nseq, path, J)
            vit()
            vms = timed(vit, 3)
            del hist
        units = wl.particle_updates()
        ach = algorithmic_ops(wl) / (kms / 1000.0) / 1e9
        vach = recursion_ops(wl) / (vms / 1000.0) / 1e9
        # fewer sequences than SMs: one block per sequence, so the SMs the
        # launch occupies bound it, not the whole GPU
        _, _, grid = abi_grid[name] if name in abi_grid else (0, 0, sms)
        occ_sms = max(1, min(sms, grid))
        peak_occ = alu_peak_gops(pk.get("sm_max_mhz", 2070.0), occ_sms)
        line = {"config": name, "workload": desc, "B": wl.B, "N": wl.N, "d": wl.d, "L": wl.L,
                "T": f"{int(wl.T.min())}..{int(wl.T.max())}" if wl.T.min() != wl.T.max() else int(wl.T[0]),
                "metric": METRIC, "value": units / (ms / 1000.0), "unit": UNIT, "ms_per_batch": ms,
                "sequences_per_s": wl.B / (ms / 1000.0),
                "roofline": {"bound": "alu", "kernel": "seq_kernel", "kernel_ms": kms, "achieved": ach,
                             "peak": peak, "unit": "Gop/s", "frac": ach / peak, "occupied_sms": occ_sms,
                             "frac_of_occupied_sms": ach / peak_occ},
                "viterbi": {"ms": vms, "achieved": vach, "frac": vach / peak, "unit": "Gop/s"},
                "cpu_baseline": cpu_baseline(wl, os.cpu_count() or 1, t_sample)}
        print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    """The oracle as it stands on the host cores: each step is a bounded
    sample of the same workload (one sequence per host thread, the first
    T_sample steps of each)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    T_sample = 6 if args.config != "C1" else 50
    B_full = args.B or DEFAULT_B[args.config]
    wl = make_workload(args.config, 0, min(threads, B_full))   # the first sequences of the workload
    T_sample = min(T_sample, int(wl.T.min()))
    from oracle import oracle as O
    O.lib()
    T = np.full(wl.B, T_sample, np.int32)

    def one():
        t0 = time.perf_counter()
        O.run_batch(wl.kind, wl.params, wl.N, wl.L, wl.step, wl.bw_rule, wl.bw_value, wl.prior,
                    wl.seed, np.arange(wl.B), wl.x0, wl.y[:, :T_sample].astype(np.float64), T,
                    nthreads=threads)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        one()
    times = [one() for _ in range(args.steps)]
    ms = 1000.0 * float(np.mean(times))
    units = float(wl.B * wl.N * wl.L * T_sample)
    value = units / (ms / 1000.0)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.config} " + CONFIGS[args.config][1] + f", B={B_full} per GPU",
                   "N": wl.N, "L": wl.L, "B": B_full,
                   "reference_step": f"{wl.B} sequences x {T_sample} steps on {threads} host threads"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": min(threads, wl.B), "kind": "oracle",
                         "sample": f"{wl.B} sequences x first {T_sample} steps per bench step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def learned_keys(log):
    """Learned L=5 vs plain L=50 on the data-association shape with the
    batched configuration's uneven lengths and on the arm shape (4096
    sequences each); the networks are trained first (round 1 on plain-run data
    only, rounds 2-3 self-distilled)."""
    from measure import learned
    out = {}
    for which, T, train_seqs in (("clutter", None, 450), ("arm", 100, 1000)):
        r = learned.compare(which, T=T, train_seqs=train_seqs, eval_seqs=4096, rounds=3, reps=1,
                            log=lambda h: log(f"[bench] learned {which} round {h['round']}: "
                                              f"mean J {h['learned_mean_J']:.2f}"))
        out[which] = {
            "workload": r["workload"],
            "speedup_learned_vs_plain": r["speedup_learned_vs_plain"],
            "sequences_per_s": {"plain_L50": r["plain"]["sequences_per_s"],
                                "learned_L5": r["learned"]["sequences_per_s"],
                                "plain_L5": r["plain_small_L"]["sequences_per_s"]},
            "mean_J": {"plain_L50": r["plain"]["mean_J"],
                       "learned_L5_plain_data": r["training"][0]["learned_mean_J"],
                       "learned_L5_self_distilled": r["learned"]["mean_J"],
                       "plain_L5": r["plain_small_L"]["mean_J"]},
            "J_gap_rel_plain_data": r["J_gap_rel_plain_data"],
            "J_gap_rel_self_distilled": r["J_gap_rel"],
            "training": [{k: h[k] for k in ("round", "data", "rows", "sequence_steps", "loss_last",
                                            "data_seconds", "train_seconds")} for h in r["training"]],
            "timing": r["timing"],
        }
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="smap", choices=["smap", "reference"])
    ap.add_argument("--config", default=DEFAULT_CONFIG, choices=sorted(CONFIGS))
    ap.add_argument("--B", type=int, default=None, help="sequences per GPU (default: the configuration's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-c5", action="store_true", help="skip the learned-proposal keys")
    ap.add_argument("--all-configs", action="store_true",
                    help="one line per workload configuration (C1-C4) instead of the bench line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.all_configs:
        return all_configs(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    from paper_2312_08684_gb300 import Estimator, _binding as abi

    def log(msg):
        if rank == 0:
            print(msg, file=sys.stderr, flush=True)

    wl = make_workload(args.config, rank, args.B)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    stream = torch.cuda.Stream()
    est = Estimator.from_workload(wl, stream=stream)
    y_dev = torch.from_numpy(wl.y).to(dev)
    path_dev = torch.empty((wl.B, wl.maxT + 1, wl.d), dtype=torch.float32, device=dev)
    J_dev = torch.empty(wl.B, dtype=torch.float64, device=dev)
    T_seq = np.ascontiguousarray(wl.T, np.int32)
    tune = None
    if not args.no_autotune:
        # every compiled launch shape on the whole batch for its first 3 steps
        chosen, ms_v = est.autotune(y_dev, sample=wl.B, steps=3)
        tune = {"chosen_variant": int(chosen), "sample": f"{wl.B} sequences x 3 steps",
                "ms_per_variant": [None if not np.isfinite(m) else float(m) for m in ms_v]}
        log(f"[bench] autotune: variant {chosen}, ms {ms_v}")
    variant, threads, _ = abi.smap_get_variant(est.h)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def device_step():
        abi.smap_run_batch(est.h, y_dev, T_seq, None, path_dev, J_dev)

    for _ in range(max(args.warmup, 3)):
        device_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    launches0 = abi.smap_kernel_launches()
    step_ms, kern_ms = [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()                       # L2 flush between timed steps (256 MB write)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ev0.record(stream)
            device_step()
            ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        kern_ms.append(abi.smap_last_kernel_ms(est.h)[0])
    torch.cuda.synchronize()
    launches = abi.smap_kernel_launches() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(float(np.mean(step_ms)), dist, dev)
    if dist:
        dist.barrier()
    units_rank = wl.particle_updates()
    value = units_rank * world / (ms / 1000.0)
    log(f"[bench] {args.steps} steps: {ms:.1f} ms per step")

    # end to end through the public call with host buffers (pinned), copies inside
    y_pin = torch.from_numpy(wl.y).pin_memory()
    path_pin = torch.empty((wl.B, wl.maxT + 1, wl.d), dtype=torch.float32).pin_memory()
    J_pin = torch.empty(wl.B, dtype=torch.float64).pin_memory()
    e2e_t = []
    for k in range(max(2, min(args.steps, 3)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        abi.smap_run_batch(est.h, y_pin, T_seq, None, path_pin, J_pin)
        if k:
            e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(float(np.mean(e2e_t)), dist, dev)

    # the recursion alone (smap_viterbi on this run's particle sets): its own
    # roofline against the same ALU peak
    hist_dev = torch.empty((wl.B, wl.maxT, wl.N, wl.d), dtype=torch.float32, device=dev)
    abi.smap_get_history(est.h, hist_dev)
    abi.smap_viterbi(est.h, hist_dev, y_dev, T_seq, None, path_dev, J_dev)
    abi.smap_debug_recursion_stats(est.h)          # counters from here on: the timed recursion runs
    vit_ms = []
    for _ in range(3):
        flush.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ev0.record(stream)
            abi.smap_viterbi(est.h, hist_dev, y_dev, T_seq, None, path_dev, J_dev)
            ev1.record(stream)
        ev1.synchronize()
        vit_ms.append(ev0.elapsed_time(ev1))
    vit_ms = max_over_ranks(float(np.mean(vit_ms)), dist, dev)
    n_ps, n_tie, n_eval = abi.smap_debug_recursion_stats(est.h)
    del hist_dev
    est.close()
    del y_dev, path_dev, J_dev, flush
    torch.cuda.empty_cache()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    pk, src = peaks()
    sm_for_peak = pk.get("sm_max_mhz", 2070.0)
    peak = alu_peak_gops(sm_for_peak, sms)
    kms = float(np.mean(kern_ms))
    achieved = algorithmic_ops(wl) / (kms / 1000.0) / 1e9
    traffic = seq_kernel_traffic(args.config, wl)
    vit_ach = recursion_ops(wl) / (vit_ms / 1000.0) / 1e9
    tlen = f"T={int(wl.T[0])}" if wl.T.min() == wl.T.max() else f"T={int(wl.T.min())}..{int(wl.T.max())}"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "sequences_per_s": wl.B * world / (ms / 1000.0),
        "config": {"workload": f"{args.config} {CONFIGS[args.config][1]}, B={wl.B} per GPU; FP32 "
                               "particles, FP64 Viterbi scores",
                   "N": wl.N, "L": wl.L, "T": tlen, "B": wl.B, "parallelism": f"sequences x{world}",
                   "kernel_variant": {"variant": int(variant), "threads": int(threads),
                                      "chosen_by": "autotune" if tune else "built-in heuristic"},
                   "l2": "flushed between timed steps (256 MB write)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "seq_kernel",
                     "kernel_ms": kms,
                     "peak_basis": f"{sms} SMs x 128 FP32 lanes x {sm_for_peak:.0f} MHz ({src} max clock)"},
        "e2e": {"value": units_rank * world / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(wl.y.nbytes),
                "d2h_bytes_per_step": int(path_pin.numel() * 4 + J_pin.numel() * 8)},
        "viterbi": {"what": "smap_viterbi alone on the same particle sets (history copy, recursion, "
                            "backtrack)", "ms": vit_ms, "achieved": vit_ach, "peak": peak, "unit": "Gop/s",
                    "frac": vit_ach / peak, "ops_per_pair": 2 * wl.d + 2,
                    "near_tie_fraction": n_tie / max(n_ps, 1),
                    "exact_scores_per_particle_step": n_eval / max(n_ps, 1)},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if tune:
        line["autotune"] = tune
    if not args.no_c5 and world == 1:
        line["learned_proposal"] = learned_keys(log)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, os.cpu_count() or 1, CONFIGS[args.config][2])
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
