"""Pins of the oracle's scenario models and RNG against things other than itself:
scipy's densities, central finite differences, published known-answer vectors
and distributional tests (CPU only)."""
import os

import numpy as np
import pytest
from scipy import special, stats

from paper_2312_08684_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _models(O):
    rng = np.random.default_rng(0)
    beacons = rng.uniform(0, 100, (3, 2))
    return {
        "ngm1d": (O.Model(1, W.ngm1d_params()), lambda r: r.normal(0, 4, 1), lambda r: r.normal(5, 3, 1)),
        "ngm1d_paper": (O.Model(1, W.ngm1d_params(True)), lambda r: r.normal(0, 4, 1), lambda r: r.normal(5, 3, 1)),
        "range": (O.Model(2, W.range_params(beacons)), lambda r: np.r_[r.uniform(20, 80, 2), r.normal(0, 1, 2)],
                  lambda r: r.uniform(5, 60, 3)),
        "clutter": (O.Model(3, W.clutter_params()), lambda r: np.r_[r.uniform(-10, 10, 2), r.normal(0, 1, 2)],
                    lambda r: r.uniform(-12, 12, 20)),
        "arm": (O.Model(4, W.arm_params()), lambda r: np.r_[r.uniform(-0.5, 0.5, 7), r.normal(0, 0.1, 7)],
                lambda r: r.normal(0, 1.0, 2)),
        "linear": (O.Model(5, W.linear_params()), lambda r: np.r_[r.normal(0, 3, 2), r.normal(0, 1, 2)],
                   lambda r: r.normal(0, 3, 2)),
        "range_zv": (O.Model(6, W.zv_params()), lambda r: r.uniform(-2, 12, 2), lambda r: r.uniform(0, 14, 3)),
        "se2_rb": (O.Model(7, W.se2_params()), lambda r: np.r_[r.uniform(-11, 11, 2), r.uniform(-4, 4)],
                   lambda r: np.r_[r.uniform(1, 25), r.uniform(-3, 3)]),
    }


def test_philox_known_answers(oracle):
    """Philox-4x32-10 against the generator's published known-answer vectors."""
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        a, b = line.split("|")
        a = [int(v, 16) for v in a.split()]
        b = [int(v, 16) for v in b.split()]
        assert list(oracle.philox4x32_10(a[:4], a[4:])) == b
        n += 1
    assert n == 3


def test_normals_are_standard_normal(oracle):
    """Box-Muller output: Kolmogorov-Smirnov against N(0,1), per coordinate slot,
    and independence of the two members of a pair (correlation ~ 0)."""
    d = 6
    z = np.array([oracle.normals(123456789, 7, t, i, d) for t in range(1, 41) for i in range(250)])
    for c in range(d):
        assert stats.kstest(z[:, c], "norm").pvalue > 1e-3
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 0.05
    assert abs(np.corrcoef(z[:, 0], z[:, 4])[0, 1]) < 0.05
    # distinct counters give distinct draws; same counter gives the same draw
    assert not np.allclose(oracle.normals(1, 0, 1, 0, 4), oracle.normals(1, 0, 1, 1, 4))
    assert np.array_equal(oracle.normals(1, 0, 1, 0, 4), oracle.normals(1, 0, 1, 0, 4))


def test_loglik_against_scipy(oracle):
    rng = np.random.default_rng(1)
    beacons = rng.uniform(0, 100, (3, 2))
    # NGM1D: z ~ N(hcoef x^2, r)
    m = oracle.Model(1, W.ngm1d_params())
    for _ in range(20):
        x, z = rng.normal(0, 5), rng.normal(5, 3)
        assert m.loglik(3, [z], [x]) == pytest.approx(stats.norm.logpdf(z, 0.05 * x * x, 1.0), rel=1e-12)
    # RANGE: product over heard beacons; NaN = not heard
    p = W.range_params(beacons)
    m = oracle.Model(2, p)
    for _ in range(20):
        x = np.r_[rng.uniform(0, 100, 2), rng.normal(0, 1, 2)]
        z = rng.uniform(0, 80, 3)
        rho = np.linalg.norm(x[:2] - beacons, axis=1)
        ref = stats.norm.logpdf(z, rho, np.sqrt(0.25)).sum()
        assert m.loglik(1, z, x) == pytest.approx(ref, rel=1e-12)
        z2 = z.copy(); z2[1:] = np.nan
        assert m.loglik(1, z2, x) == pytest.approx(stats.norm.logpdf(z[0], rho[0], 0.5), rel=1e-12)
    # CLUTTER: (1-beta)/M sum N(z_m; p, rI) + beta/area
    m = oracle.Model(3, W.clutter_params())
    for _ in range(20):
        x = np.r_[rng.uniform(-10, 10, 2), rng.normal(0, 1, 2)]
        z = rng.uniform(-12, 12, (10, 2))
        comp = stats.multivariate_normal.logpdf(z, x[:2], 0.5 * np.eye(2)) + np.log(0.8 / 10)
        ref = special.logsumexp(np.r_[comp, np.log(0.2 / 1e4)])
        assert m.loglik(1, z.ravel(), x) == pytest.approx(ref, rel=1e-12)
    # PLANAR_ARM: end effector as a sum of complex phasors
    m = oracle.Model(4, W.arm_params())
    for _ in range(20):
        x = np.r_[rng.uniform(-1, 1, 7), rng.normal(0, 1, 7)]
        e = np.sum(0.3 * np.exp(1j * np.cumsum(x[:7])))
        z = np.array([e.real, e.imag]) + rng.normal(0, 0.02, 2)
        ref = stats.multivariate_normal.logpdf(z, [e.real, e.imag], 1e-4 * np.eye(2))
        assert m.loglik(1, z, x) == pytest.approx(ref, rel=1e-10)
    # RANGE_ZV2D: the same range product for a 2-D position
    m = oracle.Model(6, W.zv_params())
    for _ in range(20):
        x = rng.uniform(-2, 12, 2)
        z = rng.uniform(0, 14, 3)
        rho = np.linalg.norm(x - W.ZV_ANCHORS, axis=1)
        assert m.loglik(1, z, x) == pytest.approx(stats.norm.logpdf(z, rho, 0.5).sum(), rel=1e-12)
        z2 = z.copy(); z2[0] = np.nan
        assert m.loglik(1, z2, x) == pytest.approx(stats.norm.logpdf(z[1:], rho[1:], 0.5).sum(), rel=1e-12)
    # SE2_RB: equal-weight mixture over the four landmarks of a range density
    # times a bearing density of the residual taken on the circle
    m = oracle.Model(7, W.se2_params())
    lm = W.SE2_LANDMARKS
    for _ in range(40):
        x = np.r_[rng.uniform(-11, 11, 2), rng.uniform(-4, 4)]
        z = np.r_[rng.uniform(1, 25), rng.uniform(-np.pi, np.pi)]
        rho = np.linalg.norm(x[:2] - lm, axis=1)
        bear = np.arctan2(x[1] - lm[:, 1], x[0] - lm[:, 0])
        res = np.angle(np.exp(1j * (z[1] - bear)))
        ref = special.logsumexp(stats.norm.logpdf(z[0], rho, 1.0) + stats.norm.logpdf(res, 0, 0.44)) - np.log(4)
        assert m.loglik(1, z, x) == pytest.approx(ref, rel=1e-12)
        # the heading does not enter the measurement
        assert m.loglik(1, z, np.r_[x[:2], x[2] + 1.0]) == pytest.approx(ref, rel=1e-12)
    assert m.loglik(1, np.array([np.nan, 0.3]), np.zeros(3)) == 0.0
    # LINEAR_GAUSS
    m = oracle.Model(5, W.linear_params())
    x = rng.normal(0, 1, 4); z = rng.normal(0, 1, 2)
    assert m.loglik(1, z, x) == pytest.approx(
        stats.multivariate_normal.logpdf(z, x[:2], 0.05 * np.eye(2)), rel=1e-12)


def test_logtrans_and_transition_against_scipy(oracle):
    rng = np.random.default_rng(2)
    m = oracle.Model(4, W.arm_params())
    q = W.arm_params()[3:17]
    for _ in range(10):
        x, f = rng.normal(0, 1, 14), rng.normal(0, 1, 14)
        assert m.logtrans(x, f) == pytest.approx(stats.multivariate_normal.logpdf(x, f, np.diag(q)), rel=1e-12)
    # constant-velocity transition = the matrix [[I, dt I], [0, I]]
    m = oracle.Model(2, W.range_params(np.zeros((3, 2))))
    F = np.block([[np.eye(2), 0.1 * np.eye(2)], [np.zeros((2, 2)), np.eye(2)]])
    x = rng.normal(0, 1, 4)
    assert np.allclose(m.transition(5, x), F @ x, rtol=0, atol=1e-15)
    # zero-velocity random walk: the identity, with density N(x; f, 0.01 I)
    m = oracle.Model(6, W.zv_params())
    x = rng.normal(0, 3, 2)
    assert np.array_equal(m.transition(7, x), x)
    f = rng.normal(0, 3, 2)
    assert m.logtrans(x, f) == pytest.approx(stats.multivariate_normal.logpdf(x, f, 0.01 * np.eye(2)), rel=1e-12)
    # SE(2) motion with constant controls: K steps of heading increment
    # 2 pi / K trace a closed regular K-gon, counter-clockwise for w > 0, whose
    # vertices lie on a circle of radius v dt / (2 sin(pi / K))
    K, dt, v = 100, 0.1, 1.0
    w = 2 * np.pi / K / dt
    p = W.se2_params(v=v, w=w, dt=dt)
    m = oracle.Model(7, p)
    x = np.array([3.0, -1.0, 0.4])
    pts = [x]
    for t in range(K):
        pts.append(m.transition(t + 1, pts[-1]))
    pts = np.array(pts)
    assert np.allclose(pts[-1, :2], pts[0, :2], atol=1e-12)
    assert pts[-1, 2] == pytest.approx(pts[0, 2] + 2 * np.pi, abs=1e-12)
    # Section V-B moves the position along the NEW heading theta_t
    step1 = pts[1, :2] - pts[0, :2]
    assert np.arctan2(step1[1], step1[0]) == pytest.approx(0.4 + w * dt, abs=1e-12)
    side = np.linalg.norm(np.diff(pts[:, :2], axis=0), axis=1)
    assert np.allclose(side, v * dt, rtol=1e-12)
    xy = pts[:-1, :2]
    area = 0.5 * np.sum(xy[:, 0] * np.roll(xy[:, 1], -1) - np.roll(xy[:, 0], -1) * xy[:, 1])
    R = v * dt / (2 * np.sin(np.pi / K))
    assert area == pytest.approx(0.5 * K * R * R * np.sin(2 * np.pi / K), rel=1e-9)
    centre = xy.mean(axis=0)
    assert np.allclose(np.linalg.norm(xy - centre, axis=1), R, rtol=1e-9)
    # NGM1D time dependence: cos(1.2 t) in the workload form, cos(1.2 (t-1)) in the paper's
    m = oracle.Model(1, W.ngm1d_params())
    assert m.transition(3, [2.0])[0] == pytest.approx(1.0 + 50.0 / 5.0 + 8 * np.cos(3.6), rel=1e-14)
    m = oracle.Model(1, W.ngm1d_params(True))
    assert m.transition(3, [2.0])[0] == pytest.approx(1.8 + 20.0 / 5.0 + 8 * np.cos(2.4), rel=1e-14)


@pytest.mark.parametrize("name", ["ngm1d", "ngm1d_paper", "range", "clutter", "arm", "linear", "range_zv",
                                  "se2_rb"])
def test_grad_loglik_finite_differences(oracle, name):
    m, xs, zs = _models(oracle)[name]
    rng = np.random.default_rng(3)
    for _ in range(10):
        x, z = xs(rng), zs(rng)
        g = m.grad_loglik(2, z, x)
        for c in range(m.d):
            hstep = 1e-6 * max(1.0, abs(x[c]))
            xp, xm = x.copy(), x.copy()
            xp[c] += hstep; xm[c] -= hstep
            fd = (m.loglik(2, z, xp) - m.loglik(2, z, xm)) / (2 * hstep)
            assert g[c] == pytest.approx(fd, rel=1e-5, abs=1e-6 * max(1.0, abs(fd)))


def test_grad_prior_mixture_and_meangrad(oracle):
    """MIXTURE = gradient of log (1/N) sum_j N(x; f_j, Q) (FD of scipy logsumexp);
    MEANGRAD = gradient of (1/N) sum_j log N(x; f_j, Q); equal for one component."""
    rng = np.random.default_rng(4)
    m = oracle.Model(5, W.linear_params())
    q = m.q
    for Np in (1, 3, 17):
        fprev = rng.normal(0, 0.3, (Np, 4))
        x = rng.normal(0, 0.3, 4)

        def mix(v):
            return special.logsumexp(stats.multivariate_normal.logpdf(fprev, v, np.diag(q))) - np.log(Np)

        def mean(v):
            return np.mean(np.atleast_1d(stats.multivariate_normal.logpdf(fprev, v, np.diag(q))))

        gm, ga = m.grad_prior(0, fprev, x), m.grad_prior(1, fprev, x)
        for c in range(4):
            e = np.zeros(4); e[c] = 1e-6
            assert gm[c] == pytest.approx((mix(x + e) - mix(x - e)) / 2e-6, rel=1e-5, abs=1e-4)
            assert ga[c] == pytest.approx((mean(x + e) - mean(x - e)) / 2e-6, rel=1e-5, abs=1e-4)
        if Np == 1:
            assert np.allclose(gm, ga, rtol=1e-14, atol=0)


def test_grad_prior_map_conditioned(oracle):
    """MAPCOND = gradient of max_j [phi_j + log N(x; f_j, Q)] (central finite
    differences of scipy densities where the best j is clear); one previous
    particle gives the mixture's gradient; a dominant phi_j selects that
    component alone."""
    rng = np.random.default_rng(6)
    m = oracle.Model(5, W.linear_params())
    q = m.q
    for Np in (1, 4, 23):
        fprev = rng.normal(0, 0.3, (Np, 4))
        phi = rng.normal(0, 2.0, Np)
        for _ in range(5):
            x = rng.normal(0, 0.3, 4)

            def env(v):
                return np.max(phi + np.atleast_1d(stats.multivariate_normal.logpdf(fprev, v, np.diag(q))))

            vals = np.sort(phi + np.atleast_1d(stats.multivariate_normal.logpdf(fprev, x, np.diag(q))))
            if Np > 1 and vals[-1] - vals[-2] < 1e-2:
                continue
            g = m.grad_prior(2, fprev, x, phi)
            for c in range(4):
                e = np.zeros(4); e[c] = 1e-7
                assert g[c] == pytest.approx((env(x + e) - env(x - e)) / 2e-7, rel=1e-5, abs=1e-4)
        if Np == 1:
            x = rng.normal(0, 0.3, 4)
            assert np.allclose(m.grad_prior(2, fprev, x, phi), m.grad_prior(0, fprev, x), rtol=1e-14, atol=0)
    fprev = rng.normal(0, 0.3, (5, 4))
    phi = np.zeros(5); phi[3] = 1e4
    x = rng.normal(0, 0.3, 4)
    assert np.allclose(m.grad_prior(2, fprev, x, phi), (fprev[3] - x) / q, rtol=1e-14, atol=0)
