"""The roofline accounting of bench.py (CPU only): the algorithmic operation
counts follow the stated per-pair figures, and a committed DRAM-traffic
summary is read back only for exactly its workload and kernel sources."""
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
    wl = b.W.make_range_cv(B=8, T=12, N=16, L=5)
    d = wl.d
    per_seq = 16 ** 2 * 12 * (5 * (8 * d + 8) + (2 * d + 2))
    assert b.algorithmic_ops(wl) == 8 * per_seq
    # the recursion: one predecessor at t = 1, N at every later step
    assert b.recursion_ops(wl) == 8 * (16 * 16 * 11 + 16) * (2 * d + 2)


def test_traffic_summary_matches_the_bench_workload():
    b = _bench()
    wl = b.make_workload(b.DEFAULT_CONFIG, 0)
    t = b.seq_kernel_traffic(b.DEFAULT_CONFIG, wl)
    # within 10 % of the algorithmic bytes sum_s T_s (4 N d + 2 N + 4 dy)
    alg = float(wl.T.sum()) * (4 * wl.N * wl.d + 2 * wl.N + 4 * wl.dy)
    if t is not None:
        assert 0.9 * alg < t < 1.1 * alg
    # any other workload has no committed traffic figure
    small = b.W.make_clutter_cv(B=8, Tmin=12, Tmax=12, N=16, L=5)
    assert b.seq_kernel_traffic(b.DEFAULT_CONFIG, small) is None


def test_traffic_summary_needs_the_current_kernel_sources(tmp_path, monkeypatch):
    b = _bench()
    wl = b.W.make_clutter_cv(B=3, Tmin=5, Tmax=9, N=16, L=5)
    prof = tmp_path / "profiles"
    prof.mkdir()
    line = (f"traffic: B={wl.B} N={wl.N} L={wl.L} T={int(wl.T.sum())} bytes_per_launch=12345 "
            f"source={b.kernel_source_sha('C3')}\n")
    (prof / "seq_kernel_clutter_cv_traffic.md").write_text(line)
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.seq_kernel_traffic("C3", wl) == 12345
    (prof / "seq_kernel_clutter_cv_traffic.md").write_text(line.replace("source=", "source=0"))
    assert b.seq_kernel_traffic("C3", wl) is None
