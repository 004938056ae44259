"""Pins of the oracle's dynamic programme (Eq. forward_recursion and the
backtracking of Section IV-B): brute-force enumeration of every path on
small supports (Theorem 1's J(s)), a hand-built backpointer table, and the
linear-Gaussian case where the MAP path tends to the Rauch-Tung-Striebel
smoother as the particle count grows (CPU only)."""
import itertools

import numpy as np
import pytest
from scipy import stats

from paper_2312_08684_gb300 import workloads as W


def _random_case(oracle, kind, params, N, T, seed):
    rng = np.random.default_rng(seed)
    m = oracle.Model(kind, params)
    x0 = rng.normal(0, 1, m.d)
    if kind == 1:
        x0 = np.array([rng.normal(0, 2)])
    hist = x0[None, None, :] + np.cumsum(rng.normal(0, 1.0, (T, N, m.d)), axis=0) * 0.5
    z = rng.normal(0, 1, (T, m.dy))
    if kind == 1:
        z = np.abs(z) * 3
    return m, x0, hist, z


@pytest.mark.parametrize("case", range(15))
def test_viterbi_equals_brute_force(oracle, case):
    """argmax over all N^T paths of J(s) (Theorem 1) equals the DP result."""
    kinds = [(1, W.ngm1d_params()), (5, W.linear_params(q=0.5, r=0.5)),
             (2, W.range_params(np.array([[0.0, 0.0], [3.0, 0.0], [0.0, 3.0]]), q=0.5, r=0.5)),
             (6, W.zv_params(np.array([[0.0, 0.0], [3.0, 0.0], [0.0, 3.0]]), q=0.5, r=0.5)),
             (7, W.se2_params(np.array([[0.0, 0.0], [3.0, 0.0], [0.0, 3.0], [3.0, 3.0]]), alpha=(5, 5, 5)))]
    kind, params = kinds[case % 5]
    N = 2 + case % 3
    T = 5 if N <= 3 else 4
    m, x0, hist, z = _random_case(oracle, kind, params, N, T, 100 + case)
    best, bestJ = None, -np.inf
    for idx in itertools.product(range(N), repeat=T):
        path = np.vstack([x0[None, :], hist[np.arange(T), list(idx)]])
        J = m.path_score(path, z)
        if J > bestJ:
            best, bestJ = idx, J
    res = oracle.viterbi_sets(kind, params, x0, hist, z)
    assert res["J"] == pytest.approx(bestJ, rel=1e-12, abs=1e-12)
    got = res["path"]
    expect = np.vstack([x0[None, :], hist[np.arange(T), list(best)]])
    assert np.array_equal(got, expect)


def test_backtrack_hand_table(oracle):
    """psi / phi_T chosen by hand; ties go to the lowest index."""
    T, N, d = 3, 3, 1
    hist = np.arange(T * N, dtype=float).reshape(T, N, d) + 100
    psi = np.array([[0, 0, 0], [2, 0, 1], [1, 2, 2]], dtype=np.int32)
    phiT = np.array([-1.0, 5.0, 5.0])          # tie between 1 and 2: pick 1
    path, idx, J = oracle.backtrack(np.array([7.0]), hist, psi, phiT)
    # i_3 = 1; i_2 = psi_3(1) = 2; i_1 = psi_2(2) = 1
    assert list(idx) == [1, 2, 1]
    assert J == 5.0
    assert list(path[:, 0]) == [7.0, hist[0, 1, 0], hist[1, 2, 0], hist[2, 1, 0]]


def test_forward_initialisation_is_joint_density(oracle):
    """phi_1(i) = log p(z_1, x_1^i | x_0^true) (single previous particle)."""
    m = oracle.Model(2, W.range_params(np.array([[0.0, 0.0], [10.0, 0.0], [0.0, 10.0]])))
    rng = np.random.default_rng(3)
    x0 = np.array([4.0, 5.0, 1.0, -1.0])
    f = m.transition(1, x0)
    x = f + rng.normal(0, 0.1, (5, 4))
    z = np.array([6.0, 7.0, np.nan])
    psi, phi = m.forward(1, z, f[None, :], np.zeros(1), x)
    assert np.all(psi == 0)
    for i in range(5):
        assert phi[i] == pytest.approx(m.loglik(1, z, x[i]) + m.logtrans(x[i], f), rel=1e-14)


def _rts(F, Q, H, R, x0, z):
    """Kalman filter from a known x_0 (zero covariance) + Rauch-Tung-Striebel pass."""
    T = z.shape[0]; n = F.shape[0]
    xf = np.zeros((T, n)); Pf = np.zeros((T, n, n)); xp = np.zeros((T, n)); Pp = np.zeros((T, n, n))
    x, P = x0.copy(), np.zeros((n, n))
    for t in range(T):
        x, P = F @ x, F @ P @ F.T + Q
        xp[t], Pp[t] = x, P
        S = H @ P @ H.T + R
        K = P @ H.T @ np.linalg.inv(S)
        x = x + K @ (z[t] - H @ x)
        P = (np.eye(n) - K @ H) @ P
        xf[t], Pf[t] = x, P
    xs = xf.copy()
    for t in range(T - 2, -1, -1):
        C = Pf[t] @ F.T @ np.linalg.inv(Pp[t + 1])
        xs[t] = xf[t] + C @ (xs[t + 1] - xp[t + 1])
    return xs


@pytest.mark.slow
def test_map_path_tends_to_rts_smoother(oracle):
    """Linear-Gaussian: the posterior over x_{1:T} is Gaussian, so its MAP is the
    RTS smoother mean, and J(RTS path) >= J(any path), the particle MAP included
    (J of the RTS path taken from scipy densities). The Stein-MAP-Seq path over
    particle supports gets closer to the smoother as N grows (mean over four
    seeded sequences; the rate is slow in a 4-D state)."""
    B, T, L, step = 4, 10, 100, 0.002
    wl = W.make_linear_gauss(B=B, T=T, N=8, L=L, step=step, q=0.01, r=0.05)
    F = np.block([[np.eye(2), 0.1 * np.eye(2)], [np.zeros((2, 2)), np.eye(2)]])
    Q = 0.01 * np.eye(4); H = np.hstack([np.eye(2), np.zeros((2, 2))]); R = 0.05 * np.eye(2)

    def J_of(x0, path, z):
        J, prev = 0.0, x0
        for t in range(len(z)):
            J += stats.multivariate_normal.logpdf(z[t], H @ path[t], R)
            J += stats.multivariate_normal.logpdf(path[t], F @ prev, Q)
            prev = path[t]
        return J

    gaps = []
    for N in (4, 32, 128):
        g = []
        for s in range(B):
            z = wl.y[s].astype(np.float64)
            res = oracle.run_sequence(wl.kind, wl.params, N, L, step, 0, 1.0, 0, 11, s, wl.x0[s], z)
            xs = _rts(F, Q, H, R, wl.x0[s], z)
            assert res["J"] <= J_of(wl.x0[s], xs, z) + 1e-9
            assert res["J"] == pytest.approx(J_of(wl.x0[s], res["path"][1:], z), rel=1e-12)
            g.append(np.sqrt(np.mean((res["path"][1:, :2] - xs[:, :2]) ** 2)))
        gaps.append(np.mean(g))
    assert gaps[0] > gaps[1] > gaps[2]
    assert gaps[2] < 0.7 * gaps[0]


def test_margins_against_direct_scipy(oracle):
    """The margin helper used by the GPU tests: best minus second best of
    phi_{t-1}(j) + log N(x_t^i; f(x_{t-1}^j), Q), computed here with scipy."""
    wl = W.make_linear_gauss(B=1, T=4, N=5)
    rng = np.random.default_rng(2)
    hist = wl.truth[0, 1:, None, :] + 0.3 * rng.normal(0, 1, (4, 5, 4))
    z = wl.y[0].astype(np.float64)
    F = np.block([[np.eye(2), 0.1 * np.eye(2)], [np.zeros((2, 2)), np.eye(2)]])
    Q = 0.01 * np.eye(4)
    got = oracle.viterbi_margins(wl.kind, wl.params, wl.x0[0], hist, z)
    assert np.all(np.isinf(got[0]))
    phi = np.array([stats.multivariate_normal.logpdf(z[0], hist[0, i, :2], 0.05 * np.eye(2))
                    + stats.multivariate_normal.logpdf(hist[0, i], F @ wl.x0[0], Q) for i in range(5)])
    for t in range(1, 4):
        S = np.array([[stats.multivariate_normal.logpdf(hist[t, i], F @ hist[t - 1, j], Q) + phi[j]
                       for j in range(5)] for i in range(5)])
        srt = np.sort(S, axis=1)
        expect = (srt[:, -1] - srt[:, -2]) / np.maximum(1.0, np.abs(srt[:, -1]))
        assert np.allclose(got[t], expect, rtol=1e-9, atol=1e-12)
        best = S.max(1)
        phi = best + np.array([stats.multivariate_normal.logpdf(z[t], hist[t, i, :2], 0.05 * np.eye(2))
                               for i in range(5)])
