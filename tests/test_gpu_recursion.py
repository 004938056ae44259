"""The recursion-only kernel behind smap_viterbi (Eq. forward_recursion and
backtracking, Section IV-B) against the oracle on identical particle sets, at
the shapes where its screen changes form: a set of fewer predecessors than
one chunk of 16 pairs, exactly one chunk, one chunk and a predecessor pair
more, odd counts (the pad predecessor), and particle counts that take each
compiled launch shape (2 particles per thread up to 512 threads, up to 1024
threads, 4 particles per thread). Sequences of one batch have different
lengths and particle counts.

Bar (as for the other recursion tests): psi identical wherever the oracle's
margin (best - second best candidate, relative to max(1, |best|)) exceeds
1e-6, J within 1e-12 relative, the MAP path element by element.
"""
import numpy as np
import pytest

from paper_2312_08684_gb300 import Estimator, workloads as W

pytestmark = pytest.mark.gpu

SPREAD = {"range": 0.3, "clutter": 0.3}


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _margins(m, x0, hist, z, phis):
    """Relative margin of every psi_t(i) on the oracle's scores, for the
    diagonal-Gaussian transitions of the constant-velocity models:
    phi_{t-1}(j) + log N(x_i; f_t(x_{t-1}^j), Q) over j, from the oracle's
    transition means and phi (the normaliser is taken from the oracle's own
    log-density at zero residual)."""
    T, N, d = hist.shape
    out = np.full((T, N), np.inf)
    qinv = 1.0 / m.q
    if N < 2:
        return out
    for t in range(2, T + 1):
        f = np.array([m.transition(t, v) for v in hist[t - 2]])
        c = m.logtrans(f[0], f[0])
        diff = hist[t - 1][:, None, :] - f[None, :, :]
        s = phis[t - 2][None, :] + c - 0.5 * np.einsum("ijc,c->ij", diff * diff, qinv)
        srt = np.sort(s, axis=1)
        out[t - 1] = (srt[:, -1] - srt[:, -2]) / np.maximum(1.0, np.abs(srt[:, -1]))
    return out


def _oracle_phis(m, x0, hist, z):
    """phi_t of every step from the oracle's forward recursion."""
    T = hist.shape[0]
    phis, phi = [], np.zeros(1)
    for t in range(1, T + 1):
        prev = x0[None, :] if t == 1 else hist[t - 2]
        f = np.array([m.transition(t, v) for v in prev])
        _, phi = m.forward(t, z[t - 1], f, phi, hist[t - 1])
        phis.append(phi)
    return phis


@pytest.mark.parametrize("name,Nmax,Nother", [("clutter", 31, 17), ("clutter", 32, 31), ("range", 33, 32),
                                              ("clutter", 35, 1), ("range", 513, 301),
                                              ("clutter", 1100, 1025)])
def test_recursion_kernel_matches_oracle(oracle, torch, name, Nmax, Nother):
    T = 5
    if name == "range":
        wl = W.make_range_cv(B=2, T=T, N=Nmax, dropout=(2, 3))
    else:
        wl = W.make_clutter_cv(B=2, Tmin=T, Tmax=T, N=Nmax)
    rng = np.random.default_rng(Nmax)
    B, d = wl.B, wl.d
    hist = (wl.truth[:, 1:, None, :] + SPREAD[name] * rng.normal(0, 1, (B, T, Nmax, d))).astype(np.float32)
    Tseq = np.array([T, T - 1], np.int32)
    Nseq = np.array([Nmax, Nother], np.int32)
    with Estimator.from_workload(wl) as est:
        path, J, psi = est.viterbi(hist, wl.y, Tseq, Nseq)
    m = oracle.Model(wl.kind, wl.params)
    for b in range(B):
        Tb, Nb = int(Tseq[b]), int(Nseq[b])
        hb = hist[b, :Tb, :Nb].astype(np.float64)
        zb = wl.y[b, :Tb].astype(np.float64)
        ref = oracle.viterbi_sets(wl.kind, wl.params, wl.x0[b], hb, zb)
        ok = _margins(m, wl.x0[b], hb, zb, _oracle_phis(m, wl.x0[b], hb, zb)) > 1e-6
        assert ok.mean() > 0.9
        assert np.array_equal(psi[b, :Tb, :Nb][ok], ref["psi"][ok]), f"sequence {b}: backpointers differ"
        assert J[b] == pytest.approx(ref["J"], rel=1e-12, abs=1e-9)
        assert np.array_equal(path[b, : Tb + 1], ref["path"].astype(np.float32)), f"sequence {b}: paths differ"
