"""The workload configurations at full size, in the launch configuration the
benchmark uses (one persistent, graph-replayed smap_run_batch), checked on
sampled sequences against the FP64 oracle:

  - the dynamic programme on the GPU's own particle sets: backpointers equal
    wherever the oracle's margin exceeds 1e-6 |score|, J to 1e-12, path equal;
  - one SVGD step re-run by the oracle from the GPU's previous particle set:
    final particles within 1e-3 relative;
  - J of the returned path re-scored by the oracle (Theorem 1's J(s));
  - every sequence finished with a finite J.
"""
import numpy as np
import pytest

from paper_2312_08684_gb300 import Estimator, workloads as W

pytestmark = pytest.mark.gpu

CONFIGS = {
    # 2-D range-only, d=4, N=256, L=30, T=200, B=1024 (the benchmark workload)
    "range_cv": (lambda: W.make_range_cv(), [0, 517, 1023], 2),
    # data association with clutter, d=4, N=512, L=30, T~U[50,400], B=4096
    "clutter_cv": (lambda: W.make_clutter_cv(), [0, 2048, 4095], 1),
    # 7-link planar arm, d=14, N=1024, L=50, T=100, B=256
    "planar_arm": (lambda: W.make_planar_arm(), [0, 255], 1),
}


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def rel_err(a, b):
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(1.0, np.sqrt(np.mean(b * b))))


@pytest.mark.parametrize("name", list(CONFIGS))
def test_full_size_config(oracle, torch, name):
    make, sample, svgd_steps = CONFIGS[name]
    wl = make()
    dev = torch.device("cuda:0")
    with Estimator.from_workload(wl) as est:
        path, J = est.run_batch(wl.y, wl.T, wl.Nseq)
        hist_d = torch.empty((wl.B, wl.maxT, wl.N, wl.d), dtype=torch.float32, device=dev)
        psi_d = torch.empty((wl.B, wl.maxT, wl.N), dtype=torch.int16, device=dev)
        from paper_2312_08684_gb300 import _binding as abi
        abi.smap_get_history(est.h, hist_d)
        abi.smap_get_backpointers(est.h, psi_d)
        hist = hist_d[sample].cpu().numpy()
        psi = psi_d[sample].cpu().numpy().view(np.uint16)
        del hist_d, psi_d
    assert np.all(np.isfinite(J)), "a sequence ended with a non-finite score"
    m = oracle.Model(wl.kind, wl.params)
    rng = np.random.default_rng(7)
    for k, b in enumerate(sample):
        T = int(wl.T[b])
        Hb = hist[k, :T].astype(np.float64)
        z = wl.y[b, :T].astype(np.float64)
        # dynamic programme on the GPU's own particle sets
        ref = oracle.viterbi_sets(wl.kind, wl.params, wl.x0[b], Hb, z)
        marg = oracle.viterbi_margins(wl.kind, wl.params, wl.x0[b], Hb, z)
        ok = marg > 1e-6
        assert np.array_equal(psi[k, :T][ok], ref["psi"][ok]), f"seq {b}: backpointers differ"
        assert J[b] == pytest.approx(ref["J"], rel=1e-12), f"seq {b}: J differs"
        assert np.array_equal(path[b, : T + 1], ref["path"].astype(np.float32)), f"seq {b}: path differs"
        # row 0 of the FP32 path is x_0 rounded; the recursion uses x_0 in FP64
        p64 = path[b, : T + 1].astype(np.float64)
        p64[0] = wl.x0[b]
        assert m.path_score(p64, z) == pytest.approx(J[b], rel=1e-12)
        # one SVGD step from the GPU's previous set, re-run in FP64
        for t in sorted(set([2] + list(rng.integers(3, T + 1, svgd_steps - 1)))):
            xprev = Hb[t - 2]
            f = np.array([m.transition(t, v) for v in xprev])
            xi = np.array([oracle.normals(wl.seed, b, t, i, wl.d) for i in range(wl.N)])
            x = f + np.sqrt(m.q) * xi
            xo, _ = m.svgd_iters(wl.prior, wl.bw_rule, wl.bw_value, t, z[t - 1], f, x, wl.L, wl.step)
            err = rel_err(Hb[t - 1], xo)
            assert err <= 1e-3, f"seq {b} step {t}: particles differ by {err:.3g}"
