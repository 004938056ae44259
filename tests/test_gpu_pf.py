"""PF-MAP-Seq on the GPU (smap_pf_run_batch) against the oracle: the bootstrap
filter's particle sets, the backpointers where unique to 1e-6, the MAP path
and its J, for both kernel variants (N <= 1024 and up to 4096), ragged N and
T, one particle, and models with missing measurements."""
import numpy as np
import pytest

from paper_2312_08684_gb300 import Estimator, workloads as W

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.sqrt(np.mean(b * b)))))


def _check(oracle, wl, T=None, Nseq=None):
    T = wl.T if T is None else np.asarray(T, np.int32)
    Nseq = wl.Nseq if Nseq is None else np.asarray(Nseq, np.int32)
    with Estimator.from_workload(wl) as est:
        path, J = est.pf_run_batch(wl.y, T, Nseq)
        hist = est.history()
        psi = est.backpointers()
    for b in range(wl.B):
        Tb, Nb = int(T[b]), int(Nseq[b])
        z = wl.y[b, :Tb].astype(np.float64)
        ref = oracle.pf_map_sequence(wl.kind, wl.params, Nb, wl.seed, b, wl.x0[b], z)
        # the filter's sets: FP32 copies of the FP64 particles
        assert _rel(hist[b, :Tb, :Nb], ref["hist"]) <= 1e-6, b
        marg = oracle.viterbi_margins(wl.kind, wl.params, wl.x0[b], ref["hist"], z)
        ok = marg > 1e-6
        assert np.array_equal(psi[b, :Tb, :Nb][ok], ref["psi"][ok]), b
        assert _rel(path[b, : Tb + 1], ref["path"]) <= 1e-5, b
        assert J[b] == pytest.approx(ref["J"], rel=1e-6), b
    return path, J


def test_pf_map_seq_matches_oracle_scenario_a(oracle):
    """Section V-A constants, N = 500 (the smallest PF size of Table Ex1)."""
    wl = W.make_ngm1d(B=3, T=25, N=500, paper_constants=True)
    _check(oracle, wl)


def test_pf_map_seq_large_n_variant(oracle):
    """N = 4096 and a ragged 1500: the four-particles-per-thread kernel."""
    wl = W.make_ngm1d(B=2, T=6, N=4096, paper_constants=True)
    _check(oracle, wl, Nseq=[4096, 1500])


@pytest.mark.parametrize("N", [1, 2, 33, 1024, 1025])
def test_pf_map_seq_particle_counts(oracle, N):
    wl = W.make_ngm1d(B=2, T=7, N=N, paper_constants=True)
    _check(oracle, wl, T=[7, 4])


@pytest.mark.parametrize("name", ["range", "range_zv", "se2", "linear"])
def test_pf_map_seq_other_models(oracle, name):
    wl = {"range": lambda: W.make_range_cv(B=2, T=12, N=300, dropout=(3, 6)),
          "range_zv": lambda: W.make_range_zv(B=2, T=12, N=300, blocked=((2, 5),)),
          "se2": lambda: W.make_se2_rb(B=2, T=12, N=300),
          "linear": lambda: W.make_linear_gauss(B=2, T=12, N=300)}[name]()
    _check(oracle, wl)


def test_pf_map_seq_is_deterministic():
    wl = W.make_ngm1d(B=4, T=20, N=700, paper_constants=True)
    with Estimator.from_workload(wl) as est:
        p1, J1 = est.pf_run_batch(wl.y)
        p2, J2 = est.pf_run_batch(wl.y)
    assert np.array_equal(p1, p2) and np.array_equal(J1, J2)
