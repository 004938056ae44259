"""The paper's own constants for its first scenario (Section V-A), on the GPU.

Growth model x_t = 0.9 x + 10 x / (1 + x^2) + 8 cos(1.2 (t - 1)) + v,
v ~ N(0, 5); measurement z_t = x_t^2 / 20 + r, r ~ N(0, 4^2); x_0 ~ N(0, 5);
SVGD step 0.005 and 100 iterations per step (the settings Section V states).

1. Parity with the oracle at these constants on a short run.
2. Accuracy where the paper reports it: the RMSE of the MAP sequence over 50
   trajectories of 100 steps (Table Ex1 lists 2.05 / 2.14 / 2.28 for
   N = 10 / 20 / 40). The paper's random draws and initialisation cannot be
   reproduced, so this is a band, not parity: the estimate must land within a
   factor of two of the published value and far below what ignoring the
   measurements gives.
"""
import numpy as np
import pytest

from paper_2312_08684_gb300 import Estimator, workloads as W

pytestmark = pytest.mark.gpu

PAPER_RMSE = {10: 2.0462, 20: 2.1447, 40: 2.2761}


def _paper_workload(B, T, N):
    return W.make_ngm1d(B=B, T=T, N=N, L=100, step=0.005, paper_constants=True)


def _rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.sqrt(np.mean(b * b)))))


def test_paper_constants_match_oracle(oracle):
    wl = _paper_workload(B=3, T=12, N=10)
    with Estimator.from_workload(wl) as est:
        path, J = est.run_batch(wl.y)
    for b in range(wl.B):
        ref = oracle.run_sequence(wl.kind, wl.params, wl.N, wl.L, wl.step, wl.bw_rule, wl.bw_value, wl.prior,
                                  wl.seed, b, wl.x0[b], wl.y[b].astype(np.float64))
        assert _rel_err(path[b], ref["path"]) <= 1e-3
        assert J[b] == pytest.approx(ref["J"], rel=1e-3)


@pytest.mark.parametrize("N", [10, 20, 40])
def test_map_sequence_rmse_in_the_papers_range(N):
    wl = _paper_workload(B=50, T=100, N=N)
    with Estimator.from_workload(wl) as est:
        path, J = est.run_batch(wl.y)
    err = path[:, 1:, 0].astype(np.float64) - wl.truth[:, 1:, 0]
    rmse = float(np.mean(np.sqrt(np.mean(err ** 2, axis=1))))    # per run, averaged over the runs
    # without the measurements: the noise-free propagation of x_0
    prior_only = np.zeros_like(wl.truth[:, :, 0])
    prior_only[:, 0] = wl.x0[:, 0]
    a, b, c, om, toff = wl.params[:5]
    for t in range(1, wl.maxT + 1):
        x = prior_only[:, t - 1]
        prior_only[:, t] = a * x + b * x / (1 + x * x) + c * np.cos(om * (t + toff))
    rmse_prior = float(np.mean(np.sqrt(np.mean((prior_only[:, 1:] - wl.truth[:, 1:, 0]) ** 2, axis=1))))
    print(f"N={N}: MAP-sequence RMSE {rmse:.4f} (paper {PAPER_RMSE[N]}), without measurements {rmse_prior:.4f}")
    assert np.all(np.isfinite(J))
    assert 0.5 * PAPER_RMSE[N] <= rmse <= 2.0 * PAPER_RMSE[N]
    assert rmse < 0.5 * rmse_prior


# ------------------------------------------------- Section V-C (range only) --
def test_range_only_zero_velocity_matches_oracle(oracle):
    """Zero-velocity range-only model with the paper's constants (Q = 0.01 I,
    sigma_z = 0.5, eps = 0.005, 100 iterations) and a blocked-anchor period
    inside the run, GPU vs oracle over a short trajectory."""
    wl = W.make_range_zv(B=2, T=40, N=20, blocked=((12, 15),))
    with Estimator.from_workload(wl) as est:
        path, J = est.run_batch(wl.y)
    for b in range(wl.B):
        ref = oracle.run_sequence(wl.kind, wl.params, wl.N, wl.L, wl.step, wl.bw_rule, wl.bw_value, wl.prior,
                                  wl.seed, b, wl.x0[b], wl.y[b].astype(np.float64))
        assert _rel_err(path[b], ref["path"]) <= 1e-3
        assert J[b] == pytest.approx(ref["J"], rel=1e-3)


@pytest.mark.parametrize("N", [20, 40])
def test_range_only_rmse_stays_bounded_through_blocking(N):
    """Six blocked periods of anchor 1 over 60 s at 10 Hz: the MAP sequence
    keeps its position error at the scale of the range noise (the paper
    reports 0.14-0.17 m on its recorded trajectories; these are seeded
    synthetic random walks, so the check is a bound, not a value)."""
    wl = W.make_range_zv(B=16, T=600, N=N)
    with Estimator.from_workload(wl) as est:
        path, J = est.run_batch(wl.y)
    err = path[:, 1:, :2].astype(np.float64) - wl.truth[:, 1:, :2]
    rmse = np.sqrt(np.mean(np.sum(err ** 2, axis=2), axis=1))
    print(f"N={N}: MAP-sequence position RMSE per run {np.round(rmse, 3)}")
    assert np.all(np.isfinite(J))
    assert float(np.mean(rmse)) < 0.5


# --------------------------------------------- Section V-B (SE(2), unknown association) --
def test_se2_range_bearing_matches_oracle(oracle):
    """SE(2) pose with constant controls, one range-bearing measurement per
    step from one of four landmarks (association marginalised), 10% outliers
    at four times the noise scale; Q, noise levels and 100 iterations as in
    Section V-B, SVGD step 1e-4 (see make_se2_rb). GPU vs oracle on a short run."""
    wl = W.make_se2_rb(B=2, T=40, N=20)
    with Estimator.from_workload(wl) as est:
        path, J = est.run_batch(wl.y)
    for b in range(wl.B):
        ref = oracle.run_sequence(wl.kind, wl.params, wl.N, wl.L, wl.step, wl.bw_rule, wl.bw_value, wl.prior,
                                  wl.seed, b, wl.x0[b], wl.y[b].astype(np.float64))
        assert _rel_err(path[b], ref["path"]) <= 1e-3
        assert J[b] == pytest.approx(ref["J"], rel=1e-3)


def test_se2_map_sequence_tracks_better_than_dead_reckoning(oracle):
    """Ten 630-step runs (the paper's Monte Carlo size): the MAP sequence
    tracks the simulated truth better than dead reckoning with the known
    controls. Its J against the truth's J under the same model (Theorem 1's
    score, the truth's from the oracle) is printed, not asserted: with a plain
    SVGD step small enough to be stable here, a particle lineage that drifted
    away is not pulled back within one step, so the MAP over the particle
    supports can score below the truth on some runs."""
    wl = W.make_se2_rb(B=10, T=630, N=20)
    with Estimator.from_workload(wl) as est:
        path, J = est.run_batch(wl.y)
    m = oracle.Model(wl.kind, wl.params)
    rm, rd, above = [], [], 0
    for b in range(wl.B):
        above += J[b] >= m.path_score(wl.truth[b], wl.y[b].astype(np.float64))
        dr = [wl.x0[b]]
        for t in range(wl.maxT):
            dr.append(m.transition(t + 1, dr[-1]))
        dr = np.array(dr)
        rm.append(np.sqrt(np.mean(np.sum((path[b, 1:, :2] - wl.truth[b, 1:, :2]) ** 2, axis=1))))
        rd.append(np.sqrt(np.mean(np.sum((dr[1:, :2] - wl.truth[b, 1:, :2]) ** 2, axis=1))))
    print(f"SE(2): MAP-sequence position RMSE {np.mean(rm):.3f} m, dead reckoning {np.mean(rd):.3f} m, "
          f"J(MAP) >= J(truth) in {above} of {wl.B} runs")
    assert np.all(np.isfinite(J))
    assert np.mean(rm) < np.mean(rd)
