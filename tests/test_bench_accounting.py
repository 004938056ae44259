"""The roofline accounting of bench.py (CPU only): the algorithmic operation
counts follow the stated per-pair figures, and the committed DRAM-traffic
summary is read back for exactly the bench workload."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_operation_counts():
    b = _bench()
    wl = b.make_workload(0, 8, 12, 16, 5)
    d = wl.d
    per_seq = 16 ** 2 * 12 * (5 * (8 * d + 8) + (2 * d + 2))
    assert b.algorithmic_ops(wl) == 8 * per_seq
    # the recursion: one predecessor at t = 1, N at every later step
    assert b.recursion_ops(wl) == 8 * (16 * 16 * 11 + 16) * (2 * d + 2)


def test_traffic_summary_matches_the_bench_workload():
    b = _bench()
    wl = b.make_workload(0, **b.WORKLOAD)
    t = b.seq_kernel_traffic(wl)
    assert t is not None and t > 0
    # within 10 % of the algorithmic bytes B T (4 N d + 2 N + 4 dy)
    alg = wl.B * wl.maxT * (4 * wl.N * wl.d + 2 * wl.N + 4 * wl.dy)
    assert 0.9 * alg < t < 1.1 * alg
    # any other workload has no committed traffic figure
    assert b.seq_kernel_traffic(b.make_workload(0, 8, 12, 16, 5)) is None
