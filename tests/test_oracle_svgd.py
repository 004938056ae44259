"""Pins of the oracle's SVGD stage (Algorithm 1 with the per-step directions of
Eqs. SVGD_initial_newupdate / SVGD_newupdate) against closed forms, library
routines and invariants (CPU only)."""
import numpy as np
import pytest
from scipy.spatial.distance import pdist

from paper_2312_08684_gb300 import workloads as W


@pytest.mark.parametrize("N,d", [(2, 1), (3, 2), (4, 3), (5, 1), (6, 4), (33, 4), (64, 14)])
def test_median_matches_numpy(oracle, N, d):
    """Median of the N(N-1)/2 squared distances: numpy.median over scipy pdist
    (covers odd and even pair counts)."""
    x = np.random.default_rng(N * 10 + d).normal(0, 1, (N, d))
    assert oracle.median_sqdist(x) == pytest.approx(np.median(pdist(x, "sqeuclidean")), rel=1e-14)
    assert oracle.bandwidth(x, 3.0) == pytest.approx(
        3.0 * np.median(pdist(x, "sqeuclidean")) / np.log(N), rel=1e-14)


def test_bandwidth_degenerate(oracle):
    assert oracle.bandwidth(np.zeros((1, 4))) == 1.0
    assert oracle.bandwidth(np.zeros((5, 2))) == 1.0     # all distances zero


def _lin_model(oracle, q, r):
    return oracle.Model(5, W.linear_params(q=q, r=r))


def test_single_particle_is_gradient_ascent_closed_form(oracle):
    """N=1: kappa(x,x)=1 and grad kappa=0, so SVGD is gradient ascent on
    log p(z, x | f). On the linear-Gaussian model that is
    x_L = x* + (I - eps A)^L (x_0 - x*),  A = H^T R^-1 H + Q^-1,
    x* = A^-1 (H^T R^-1 z + Q^-1 f)."""
    q, r, eps, L = 0.04, 0.1, 0.05, 37
    m = _lin_model(oracle, q, r)
    rng = np.random.default_rng(7)
    H = np.hstack([np.eye(2), np.zeros((2, 2))])
    Qi = np.eye(4) / q
    A = H.T @ H / r + Qi
    for prior in (0, 1):
        f = rng.normal(0, 1, 4)
        z = rng.normal(0, 1, 2)
        x0 = f + rng.normal(0, 0.3, 4)
        xs = np.linalg.solve(A, H.T @ z / r + Qi @ f)
        expect = xs + np.linalg.matrix_power(np.eye(4) - eps * A, L) @ (x0 - xs)
        got, h = m.svgd_iters(prior, 0, 1.0, 2, z, f[None, :], x0[None, :], L, eps)
        assert np.allclose(got[0], expect, rtol=1e-12, atol=1e-12)
        assert np.all(h == 1.0)


def test_two_particles_pure_repulsion_closed_form(oracle):
    """A flat target (huge q and r) leaves only the kernel-gradient term.
    With two particles a, b: h = |a-b|^2 / log 2 (one pair), and each moves by
    eps * (1/2) * kappa(a,b) * (2/h) * (a - b) along a-b, away from the other."""
    m = _lin_model(oracle, 1e30, 1e30)
    a, b = np.array([0.3, -0.2, 0.1, 0.0]), np.array([-0.1, 0.4, 0.2, 0.5])
    eps = 0.01
    s2 = np.sum((a - b) ** 2)
    h = s2 / np.log(2.0)
    k = np.exp(-s2 / h)
    got, hh = m.svgd_iters(0, 0, 1.0, 2, np.zeros(2), np.zeros((1, 4)), np.stack([a, b]), 1, eps)
    assert hh[0] == pytest.approx(h, rel=1e-14)
    assert np.allclose(got[0], a + eps * 0.5 * k * (2 / h) * (a - b), rtol=0, atol=1e-15)
    assert np.allclose(got[1], b + eps * 0.5 * k * (2 / h) * (b - a), rtol=0, atol=1e-15)
    assert np.sum((got[0] - got[1]) ** 2) > s2                      # repulsive


def test_repulsion_preserves_mean_and_drive_is_kernel_weighted(oracle):
    """Sum over i of the repulsive term vanishes (antisymmetric in i,k), so for a
    flat target the particle mean is unchanged after any number of iterations."""
    m = _lin_model(oracle, 1e30, 1e30)
    x = np.random.default_rng(8).normal(0, 1, (17, 4))
    got, _ = m.svgd_iters(0, 0, 1.0, 2, np.zeros(2), np.zeros((1, 4)), x, 5, 0.05)
    assert np.allclose(got.mean(0), x.mean(0), rtol=0, atol=1e-13)
    assert not np.allclose(got, x)


def test_permutation_equivariance(oracle):
    """Reordering the particles (and the previous set) reorders the result."""
    wl = W.make_range_cv(B=1, T=3, N=24, L=1)
    m = oracle.Model(wl.kind, wl.params)
    rng = np.random.default_rng(9)
    xprev = wl.truth[0, 1] + rng.normal(0, 0.2, (24, 4))
    fprev = np.array([m.transition(2, v) for v in xprev])
    x = fprev + rng.normal(0, 0.1, (24, 4))
    z = wl.y[0, 1].astype(np.float64)
    p1, p2 = rng.permutation(24), rng.permutation(24)
    a, ha = m.svgd_iters(0, 0, 1.0, 2, z, fprev, x, 3, 0.005)
    b, hb = m.svgd_iters(0, 0, 1.0, 2, z, fprev[p2], x[p1], 3, 0.005)
    assert np.allclose(a[p1], b, rtol=1e-12, atol=1e-12)
    assert np.allclose(ha, hb, rtol=1e-13)


def test_svgd_fixed_point_on_linear_gaussian(oracle):
    """Linear score g_k = -A (x_k - x*): at a stationary point of the SVGD map,
    summing the direction over i cancels the repulsion (antisymmetric), so the
    kernel-weighted mean sum_k c_k x_k / sum_k c_k with c_k = sum_i kappa_ik
    equals the Gaussian posterior mode x*."""
    q, r, hfix = 0.04, 0.1, 10.0
    m = _lin_model(oracle, q, r)
    rng = np.random.default_rng(10)
    f = rng.normal(0, 1, 4); z = rng.normal(0, 1, 2)
    H = np.hstack([np.eye(2), np.zeros((2, 2))])
    A = H.T @ H / r + np.eye(4) / q
    xs = np.linalg.solve(A, H.T @ z / r + f / q)
    x = f + rng.normal(0, 0.2, (32, 4))
    got, _ = m.svgd_iters(0, 2, hfix, 2, z, f[None, :], x, 4000, 0.01)   # fixed h
    # distance from stationarity: the size of the next direction
    again, _ = m.svgd_iters(0, 2, hfix, 2, z, f[None, :], got, 1, 0.01)
    resid = np.abs(again - got).max() / 0.01
    assert resid < 1e-3
    D2 = np.sum((got[:, None, :] - got[None, :, :]) ** 2, axis=-1)
    c = np.exp(-D2 / hfix).sum(0)
    err = np.abs((c[:, None] * got).sum(0) / c.sum() - xs).max()
    assert err < 1e-2 * resid
    # the unweighted mean is measurably off: the identity is specific to c_k
    assert np.abs(got.mean(0) - xs).max() > 10 * err


# ----------------------------------------------- kernels of the ablation ----
def _kernel_value(kernel, a, b, h):
    """The kernels' definitions (RBF, IMQ with c = 1 and exponent -1/2,
    Matern 3/2 with length scale sqrt(h)), for finite differences."""
    r2 = float(np.sum((a - b) ** 2))
    if kernel == 1:
        return (1.0 + r2 / h) ** -0.5
    if kernel == 2:
        s = np.sqrt(3.0 * r2 / h)
        return (1.0 + s) * np.exp(-s)
    return np.exp(-r2 / h)


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_two_particles_repulsion_is_the_kernel_gradient(oracle, kernel):
    """On a flat target (huge q and r) particle a moves by eps/2 times the
    gradient of k(x_b, a) with respect to x_b: checked against central finite
    differences of the kernel's definition, so the oracle's analytic gradient
    of each kernel is pinned."""
    m = _lin_model(oracle, 1e30, 1e30)
    a, b = np.array([0.3, -0.2, 0.1, 0.0]), np.array([-0.1, 0.4, 0.2, 0.5])
    eps = 0.01
    h = np.sum((a - b) ** 2) / np.log(2.0)     # the median rule with one pair
    got, hh = m.svgd_iters(0, 0, 1.0, 2, np.zeros(2), np.zeros((1, 4)), np.stack([a, b]), 1, eps, kernel=kernel)
    assert hh[0] == pytest.approx(h, rel=1e-14)
    step = 1e-6
    fd = np.array([(_kernel_value(kernel, b + step * e, a, h) - _kernel_value(kernel, b - step * e, a, h)) / (2 * step)
                   for e in np.eye(4)])
    assert np.allclose(got[0] - a, eps * 0.5 * fd, rtol=1e-7, atol=1e-14)
    assert np.allclose(got[1] - b, -(got[0] - a), rtol=1e-12, atol=1e-15)   # equal and opposite
    assert np.sum((got[0] - got[1]) ** 2) > np.sum((a - b) ** 2)             # repulsive


@pytest.mark.parametrize("kernel", [1, 2])
def test_other_kernels_keep_the_mean_and_weight_the_drive(oracle, kernel):
    """Radial kernels: the repulsive sum is antisymmetric (flat target keeps the
    particle mean); on a linear-Gaussian target one particle alone is plain
    gradient ascent, as with the RBF kernel (k(x, x) = 1, zero gradient)."""
    m = _lin_model(oracle, 1e30, 1e30)
    x = np.random.default_rng(8).normal(0, 1, (17, 4))
    got, _ = m.svgd_iters(0, 0, 1.0, 2, np.zeros(2), np.zeros((1, 4)), x, 5, 0.05, kernel=kernel)
    assert np.allclose(got.mean(0), x.mean(0), rtol=0, atol=1e-13)
    assert not np.allclose(got, x)
    m2 = _lin_model(oracle, 0.01, 0.05)
    x1 = np.array([[0.2, -0.1, 0.3, 0.05]])
    z = np.array([0.1, -0.2]); fprev = np.zeros((1, 4))
    r_rbf, _ = m2.svgd_iters(0, 0, 1.0, 2, z, fprev, x1, 3, 0.002)
    r_k, _ = m2.svgd_iters(0, 0, 1.0, 2, z, fprev, x1, 3, 0.002, kernel=kernel)
    assert np.array_equal(r_rbf, r_k)


def test_single_particle_priors_agree_over_a_run(oracle):
    """With one particle every step's previous set has one member, so the
    mixture, mean-gradient and MAP-conditioned priors give the same run."""
    wl = W.make_range_cv(B=1, T=10, N=1, L=5)
    z = wl.y[0].astype(np.float64)
    runs = [oracle.run_sequence(wl.kind, wl.params, 1, wl.L, wl.step, wl.bw_rule, wl.bw_value, prior,
                                wl.seed, 0, wl.x0[0], z) for prior in (0, 1, 2)]
    for r in runs[1:]:
        assert np.allclose(r["path"], runs[0]["path"], rtol=1e-13, atol=0)
        assert r["J"] == pytest.approx(runs[0]["J"], rel=1e-13)
