"""Pins of the oracle's PF-MAP-Seq (the particle-filter comparison method of
Section V, Godsill, Doucet and West 2001): stratified resampling recomputed from
scipy densities, the propagation rule, the uniform-weight and single-particle
special cases, and the MAP over the filter's supports by brute force (CPU only)."""
import itertools

import numpy as np
import pytest
from scipy import stats

from paper_2312_08684_gb300 import workloads as W


def test_uniforms_are_uniform(oracle):
    u = np.array([oracle.uniform(99, 3, t, i) for t in range(1, 21) for i in range(500)])
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    assert np.all((u > 0) & (u < 1))
    # a different stream from the normals' counters
    assert oracle.uniform(99, 3, 5, 7) != oracle.uniform(99, 3, 5, 8)


def test_stratified_resampling_from_scipy_weights(oracle):
    """Linear-Gaussian model: the weights of step t-1 recomputed with scipy's
    density; every ancestor is the stratum's interval C_{j-1} <= u_i < C_j, and
    the offspring counts stay within 2 of N w_j (the stratified bound)."""
    wl = W.make_linear_gauss(B=1, T=6, N=300)
    N, seed, seq = 300, 17, 2
    z = wl.y[0].astype(np.float64)
    hist, anc = oracle.pf_sets(wl.kind, wl.params, N, seed, seq, wl.x0[0], z)
    r = wl.params[5]
    for t in range(2, 7):
        prev = hist[t - 2]
        lw = stats.multivariate_normal.logpdf(prev[:, :2], mean=z[t - 2], cov=r * np.eye(2))
        w = np.exp(lw - lw.max()); w /= w.sum()
        C = np.cumsum(w)
        u = (np.arange(N) + np.array([oracle.uniform(seed, seq, t, i) for i in range(N)])) / N
        expect = np.minimum(np.searchsorted(C, u, side="right"), N - 1)
        margin = np.min(np.abs(C[:, None] - u[None, :]), axis=0)
        ok = margin > 1e-12
        assert np.array_equal(anc[t - 1][ok], expect[ok])
        counts = np.bincount(anc[t - 1], minlength=N)
        assert np.all(np.abs(counts - N * w) < 2.0)


def test_propagation_rule(oracle):
    """x_t^i = f_t(x_{t-1}^{a_i}) + sqrt(q) (.) xi(seed, seq, t, i)."""
    wl = W.make_range_cv(B=1, T=5, N=64)
    m = oracle.Model(wl.kind, wl.params)
    seed, seq = 5, 1
    hist, anc = oracle.pf_sets(wl.kind, wl.params, 64, seed, seq, wl.x0[0], wl.y[0].astype(np.float64))
    sq = np.sqrt(m.q)
    for i in range(64):
        assert np.allclose(hist[0, i], m.transition(1, wl.x0[0]) + sq * oracle.normals(seed, seq, 1, i, 4),
                           rtol=0, atol=1e-12)
    for t in range(2, 6):
        for i in range(64):
            f = m.transition(t, hist[t - 2, anc[t - 1, i]])
            assert np.allclose(hist[t - 1, i], f + sq * oracle.normals(seed, seq, t, i, 4), rtol=0, atol=1e-12)


def test_equal_weights_keep_every_particle(oracle):
    """No measurement at all (every anchor silent): the weights are equal and
    stratified resampling gives particle i the ancestor i."""
    wl = W.make_range_zv(B=1, T=8, N=50, blocked=None)
    z = np.full_like(wl.y[0], np.nan, dtype=np.float64)
    hist, anc = oracle.pf_sets(wl.kind, wl.params, 50, 3, 0, wl.x0[0], z)
    for t in range(2, 9):
        assert np.array_equal(anc[t - 1], np.arange(50))


def test_single_particle_is_a_sampled_trajectory(oracle):
    wl = W.make_ngm1d(B=1, T=12, N=1)
    z = wl.y[0].astype(np.float64)
    res = oracle.pf_map_sequence(wl.kind, wl.params, 1, 8, 0, wl.x0[0], z)
    assert np.all(res["anc"] == 0)
    m = oracle.Model(wl.kind, wl.params)
    assert np.array_equal(res["path"][1:, 0], res["hist"][:, 0, 0])
    assert res["J"] == pytest.approx(m.path_score(res["path"], z), rel=1e-12)


@pytest.mark.parametrize("kind_name", ["ngm1d", "range_zv"])
def test_pf_map_is_the_best_path_over_the_filter_supports(oracle, kind_name):
    """Brute force over all N^T paths of the filter's sets (Theorem 1's J)."""
    wl = {"ngm1d": lambda: W.make_ngm1d(B=1, T=5, N=4),
          "range_zv": lambda: W.make_range_zv(B=1, T=5, N=4, blocked=((1, 2),))}[kind_name]()
    z = wl.y[0].astype(np.float64)
    res = oracle.pf_map_sequence(wl.kind, wl.params, 4, 21, 0, wl.x0[0], z)
    m = oracle.Model(wl.kind, wl.params)
    best = -np.inf
    for idx in itertools.product(range(4), repeat=5):
        path = np.vstack([wl.x0[0][None, :], res["hist"][np.arange(5), list(idx)]])
        best = max(best, m.path_score(path, z))
    assert res["J"] == pytest.approx(best, rel=1e-12)


def test_pf_sets_have_near_tied_predecessors(oracle):
    """Why the recursion needs FP64 on particle-filter sets: at N = 2000 the
    filter samples the smooth maximum of phi_{t-1}(j) + log p(x_i | x_{t-1}^j)
    densely, so the best and second-best predecessor of a particle are
    typically 1e-6 nats apart, far below FP32's resolution of scores of
    magnitude 10-100 (scenario A constants, exact FP64 scores)."""
    wl = W.make_ngm1d(B=1, T=8, N=2000, paper_constants=True)
    z = wl.y[0].astype(np.float64)
    hist, _ = oracle.pf_sets(wl.kind, wl.params, 2000, wl.seed, 0, wl.x0[0], z)
    a, b, c, om, toff, q, r, hc = wl.params
    x = hist[:, :, 0]
    ll = -0.5 * (z[:, :1] - hc * x * x) ** 2 / r - 0.5 * np.log(2 * np.pi * r)

    def f(v, t):
        return a * v + b * v / (1 + v * v) + c * np.cos(om * (t + toff))

    phi = ll[0] - 0.5 * (x[0] - f(wl.x0[0, 0], 1)) ** 2 / q - 0.5 * np.log(2 * np.pi * q)
    gaps = []
    for t in range(2, 9):
        S = phi[None, :] - 0.5 * (x[t - 1][:, None] - f(x[t - 2], t)[None, :]) ** 2 / q
        srt = np.sort(S, axis=1)
        gaps.append(srt[:, -1] - srt[:, -2])
        phi = ll[t - 1] - 0.5 * np.log(2 * np.pi * q) + srt[:, -1]
    gaps = np.concatenate(gaps)
    assert np.median(gaps) < 1e-4
    assert np.mean(gaps < 1e-4) > 0.5


def test_pf_map_beats_every_filter_lineage(oracle):
    """Every ancestral lineage of the filter is a path through its supports, so
    its J (Theorem 1) cannot exceed the MAP sequence's."""
    wl = W.make_range_cv(B=1, T=15, N=200, dropout=(4, 8))
    z = wl.y[0].astype(np.float64)
    res = oracle.pf_map_sequence(wl.kind, wl.params, 200, 4, 0, wl.x0[0], z)
    m = oracle.Model(wl.kind, wl.params)
    for i in range(0, 200, 17):
        idx = [i]
        for t in range(14, 0, -1):
            idx.append(res["anc"][t, idx[-1]])
        idx = idx[::-1]
        path = np.vstack([wl.x0[0][None, :], res["hist"][np.arange(15), idx]])
        assert m.path_score(path, z) <= res["J"] + 1e-9 * abs(res["J"])
