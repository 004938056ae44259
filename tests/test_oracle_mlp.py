"""Pins of the oracle's learned-proposal pieces (CPU): the perceptron's
gradient against central finite differences, its tanh-form GELU against the
exact x Phi(x) within the approximation's known error, Adam's first step and
convergence on a quadratic, and the proposal features against direct
recomputations (complex-phasor kinematics, numpy sorting)."""
import numpy as np
import pytest
from scipy import stats

from paper_2312_08684_gb300 import workloads as W


def _random_mlp(oracle, n_in, H, n_out, seed):
    rng = np.random.default_rng(seed)
    n = oracle.mlp_nparams(n_in, H, n_out)
    return rng.normal(0, 0.5, n)


def test_gradient_matches_finite_differences(oracle):
    n_in, H, n_out = 5, 7, 3
    W = _random_mlp(oracle, n_in, H, n_out, 1)
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (6, n_in))
    T = rng.normal(0, 1, (6, n_out))
    loss, G = oracle.mlp_loss_grad(n_in, H, n_out, W, X, T)
    Y = oracle.mlp_forward(n_in, H, n_out, W, X)
    assert loss == pytest.approx(np.mean((Y - T) ** 2), rel=1e-13)
    for k in rng.choice(len(W), 40, replace=False):
        e = np.zeros_like(W); e[k] = 1e-6
        fd = (oracle.mlp_loss_grad(n_in, H, n_out, W + e, X, T)[0]
              - oracle.mlp_loss_grad(n_in, H, n_out, W - e, X, T)[0]) / 2e-6
        assert G[k] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_gelu_against_exact_form(oracle):
    """A 1-1-1-1 network with unit weights computes gelu(gelu(x)); one hidden
    layer with an identity-like output recovers gelu(x) = x Phi(x) up to the
    tanh approximation's error (below 1e-3 everywhere)."""
    # W1=1, b1=0, W2=1, b2=0, W3=1, b3=0
    W = np.array([1.0, 0.0, 1.0, 0.0, 1.0, 0.0])
    xs = np.linspace(-6, 6, 241)
    y = oracle.mlp_forward(1, 1, 1, W, xs[:, None])[:, 0]
    exact = lambda v: v * stats.norm.cdf(v)
    assert np.max(np.abs(y - exact(exact(xs)))) < 2e-3
    assert abs(y[-1] - exact(exact(6.0))) < 1e-6        # identity far right
    assert abs(y[0]) < 1e-6                              # zero far left


def test_adam_first_step_and_convergence(oracle):
    theta = np.array([1.0, -2.0, 0.5]); g = np.array([0.3, -4.0, 1e-3])
    m = np.zeros(3); v = np.zeros(3)
    t0 = theta.copy()
    oracle.adam(theta, g, m, v, 1, 0.01)
    # bias-corrected moments equal g and g^2 after one step
    assert np.allclose(theta, t0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    # a convex quadratic: Adam settles at the minimiser
    c = np.array([3.0, -1.0, 2.0]); a = np.array([1.0, 10.0, 0.1])
    theta = np.zeros(3); m = np.zeros(3); v = np.zeros(3)
    for t in range(1, 6001):
        oracle.adam(theta, 2 * a * (theta - c), m, v, t, 0.05 if t < 4000 else 0.005)
    assert np.allclose(theta, c, atol=2e-2)


def test_features_arm_and_clutter(oracle):
    rng = np.random.default_rng(3)
    p = W.arm_params()
    u = np.r_[rng.uniform(-1, 1, 7), rng.normal(0, 1, 7)]
    z = rng.normal(0, 1, 2)
    f = oracle.proposal_features(4, p, u, z)
    e = np.sum(0.3 * np.exp(1j * np.cumsum(u[:7])))
    g = oracle.Model(4, p).grad_loglik(1, z, u)          # pinned by finite differences
    assert np.allclose(f, np.r_[u, z, z - [e.real, e.imag], g[:7]], rtol=0, atol=1e-9)
    pc = W.clutter_params()
    u = np.r_[rng.normal(0, 3, 2), rng.normal(0, 1, 2)]
    z = rng.uniform(-10, 10, (10, 2))
    f = oracle.proposal_features(3, pc, u, z.ravel())
    rel = z - u[:2]
    order = np.argsort(np.sum(rel ** 2, 1), kind="stable")
    g = oracle.Model(3, pc).grad_loglik(1, z.ravel(), u)
    assert np.allclose(f, np.r_[u[2:], rel[order].ravel(), g[:2]], rtol=0, atol=1e-12)
    pr = W.range_params(np.zeros((3, 2)))
    z = np.array([5.0, np.nan, 7.0])
    f = oracle.proposal_features(2, pr, u, z)
    g = oracle.Model(2, pr).grad_loglik(1, z, u)
    assert np.allclose(f, np.r_[u, 5.0, 0.0, 7.0, 1.0, 0.0, 1.0, g])
