"""The seeded input generators of the paper-shaped scenarios produce what their
descriptions state (CPU only): the blocked-anchor periods of the zero-velocity
range model, the noise levels, the SE(2) motion with its controls, wrapped
bearings and the outlier rate."""
import numpy as np
import pytest

from paper_2312_08684_gb300 import workloads as W


def test_range_zv_blocking_and_noise():
    wl = W.make_range_zv(B=8, T=600, N=20)
    assert wl.y.shape == (8, 600, 3) and wl.truth.shape == (8, 601, 2)
    blocked = np.zeros(600, bool)
    for t0, n in W.ZV_BLOCKED:
        blocked[t0:t0 + n] = True
    for s in range(wl.B):
        assert np.array_equal(np.isnan(wl.y[s, :, 0]), blocked)
        assert not np.isnan(wl.y[s, :, 1:]).any()
    # zero-velocity random walk with Q = 0.01 I; ranges with sd 0.5
    dx = np.diff(wl.truth, axis=1).ravel()
    assert np.std(dx) == pytest.approx(0.1, rel=0.03)
    rho = np.linalg.norm(wl.truth[:, 1:, None, :] - W.ZV_ANCHORS[None, None], axis=3)
    res = (wl.y - rho)[~np.isnan(wl.y)]
    assert np.std(res) == pytest.approx(0.5, rel=0.03)
    assert abs(np.mean(res)) < 0.02
    # the blocking lengths are the printed durations at 10 Hz
    assert [n / 10 for _, n in W.ZV_BLOCKED] == [2.5, 5.0, 4.0, 4.0, 3.0, 3.5]


def test_se2_rb_motion_and_measurements():
    wl = W.make_se2_rb(B=6, T=630, N=20)
    p = wl.params
    dt, q, v, w = p[0], p[1:4], p[6], p[7]
    assert np.allclose(q, [(0.3 * dt) ** 2, (0.3 * dt) ** 2, (0.105 * dt) ** 2])
    assert p[4] == pytest.approx(1.0) and p[5] == pytest.approx(0.44 ** 2)
    # heading advances by w dt plus noise of sd 0.105 dt
    dth = np.diff(wl.truth[:, :, 2], axis=1).ravel()
    assert np.mean(dth) == pytest.approx(w * dt, abs=3e-4)
    assert np.std(dth) == pytest.approx(0.105 * dt, rel=0.05)
    # the position moves along the new heading by v dt (plus noise)
    step = np.diff(wl.truth[:, :, :2], axis=1)
    along = step[..., 0] * np.cos(wl.truth[:, 1:, 2]) + step[..., 1] * np.sin(wl.truth[:, 1:, 2])
    assert np.mean(along) == pytest.approx(v * dt, rel=0.02)
    # about one lap of the 10 m circle: 630 w dt = 6.3 rad, with heading noise
    # of sd 0.0105 sqrt(630) = 0.26 per run (0.11 on the mean of six)
    assert np.mean(wl.truth[:, -1, 2] - wl.truth[:, 0, 2]) == pytest.approx(630 * w * dt, abs=0.35)
    # bearings wrapped into [-pi, pi]; ranges positive on average
    assert np.all(np.abs(wl.y[..., 1]) <= np.pi + 1e-6)
    assert np.mean(wl.y[..., 0]) > 0


def test_se2_rb_outlier_rate():
    """Residual of each measurement against its nearest-consistent landmark:
    the share beyond 3 sd is about 0.1 P(|N(0, 16)| > 3) + 0.9 P(|N(0, 1)| > 3)."""
    wl = W.make_se2_rb(B=20, T=630, N=20)
    lm = W.SE2_LANDMARKS
    pos = wl.truth[:, 1:, :2]
    rho = np.linalg.norm(pos[:, :, None, :] - lm[None, None], axis=3)
    bear = np.arctan2(pos[..., None, 1] - lm[:, 1], pos[..., None, 0] - lm[:, 0])
    er = (wl.y[..., None, 0] - rho) / 1.0
    eb = np.angle(np.exp(1j * (wl.y[..., None, 1] - bear))) / 0.44
    # the generating landmark is the one whose residuals are smallest
    k = np.argmin(er ** 2 + eb ** 2, axis=2)
    r = np.take_along_axis(er, k[..., None], axis=2)[..., 0]
    from scipy import stats
    expect = 0.1 * 2 * stats.norm.sf(3 / 4) + 0.9 * 2 * stats.norm.sf(3)
    frac = np.mean(np.abs(r) > 3)
    # the nearest-landmark choice mislabels a few outliers, so only a band
    assert 0.5 * expect < frac < 1.5 * expect
