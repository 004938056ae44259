"""Seeded synthetic workloads shaped like the paper's scenarios.

This module only makes inputs: the model kind and its parameter vector, the
initial states x_0 and the observation sequences z_{1:T}. It holds none of the
estimator's arithmetic (no SVGD, no bandwidth, no recursion). To simulate the
ground-truth trajectories it restates each scenario's forward map in numpy
(a copy of the model equations used only to draw observations).

Workloads (sizes can be shrunk for tests; the default sizes are the full ones):
  ngm1d       1-D nonstationary growth model, sign-ambiguous z = x^2/20 + w,
              N=32, L=50, T=50, one sequence.                       (Section V-A form)
  range_cv    2-D range-only localisation, constant velocity d=4, three beacons
              in [0,100]^2, beacons 2 and 3 silent for steps 60..120,
              N=256, L=30, T=200, B=1024.                           (Section V-C form)
  clutter_cv  unknown data association: 10 points per step, one true (20%
              missed) and clutter uniform in [-50,50]^2, N=512, L=30,
              T ~ U[50,400], B=4096.                                 (Section V-B form)
  planar_arm  7-link planar chain (links 0.3 m), 14-D state, 2-D end effector,
              N=1024, L=50, T=100, B=256.                           (Section V-D form)
  linear_gauss constant velocity with direct position measurements: the
              linear-Gaussian case used by the smoother check.
  range_zv    2-D position without a motion prior (zero-velocity random walk,
              q = (1.0 * 0.1)^2), range-only to 3 anchors (sigma 0.5), anchor 1
              silent in six periods of 25-50 steps, T=600 at 10 Hz, N=40,
              L=100.                                                 (Section V-C form)
  se2_rb      pose on SE(2) with constant controls (1 m/s, 0.1 rad/s: one lap
              of a 10 m circle in 630 steps), one range-bearing measurement per
              step from one of four landmarks with unknown association, 10%
              outliers with four times the noise scale, T=630, N=20, L=100.
                                                                     (Section V-B form)
Parameter-vector layouts are the ones documented in include/smap.h.
"""
from __future__ import annotations

import dataclasses

import numpy as np

BASE_SEED = 20231208

MODEL_NGM1D, MODEL_RANGE_CV2D, MODEL_CLUTTER_CV2D, MODEL_PLANAR_ARM, MODEL_LINEAR_GAUSS = 1, 2, 3, 4, 5
MODEL_RANGE_ZV2D = 6
MODEL_SE2_RB = 7
BW_MEDIAN_ITER, BW_MEDIAN_STEP, BW_FIXED = 0, 1, 2
PRIOR_MIXTURE, PRIOR_MEANGRAD, PRIOR_MAPCOND = 0, 1, 2


@dataclasses.dataclass
class Workload:
    name: str
    kind: int
    params: np.ndarray        # float64 parameter vector (layout per model)
    d: int
    dy: int
    N: int                    # particles (maximum over the batch)
    L: int                    # SVGD iterations per step
    step: float               # SVGD step size epsilon
    bw_rule: int
    bw_value: float
    prior: int
    seed: int                 # estimator RNG seed (particle initialisation)
    x0: np.ndarray            # [B][d] float64, the known initial state
    y: np.ndarray             # [B][maxT][dy] float32 observations (NaN = not observed)
    T: np.ndarray             # [B] int32 sequence lengths
    Nseq: np.ndarray          # [B] int32 particles per sequence
    truth: np.ndarray         # [B][maxT+1][d] float64 simulated states
    kernel: int = 0           # Stein kernel: 0 RBF, 1 IMQ, 2 Matern 3/2

    @property
    def B(self) -> int:
        return int(self.x0.shape[0])

    @property
    def maxT(self) -> int:
        return int(self.y.shape[1])

    def pair_evals(self) -> float:
        """RBF pair evaluations of a whole run: sum_s N_s^2 L T_s."""
        return float(np.sum(self.Nseq.astype(np.float64) ** 2 * self.L * self.T))

    def particle_updates(self) -> float:
        """SVGD particle updates of a whole run: sum_s N_s L T_s."""
        return float(np.sum(self.Nseq.astype(np.float64) * self.L * self.T))

    def subset(self, idx) -> "Workload":
        idx = np.asarray(idx)
        T = self.T[idx]
        mt = int(T.max())
        return dataclasses.replace(
            self, x0=self.x0[idx].copy(), y=np.ascontiguousarray(self.y[idx, :mt]),
            T=T.copy(), Nseq=self.Nseq[idx].copy(), truth=self.truth[idx, : mt + 1].copy())


def _rng(*key):
    return np.random.default_rng([BASE_SEED, *[int(k) for k in key]])


# ---------------------------------------------------------------- ngm1d ----
def ngm1d_params(paper_constants: bool = False) -> np.ndarray:
    if paper_constants:   # Section V-A: 0.9x + 10x/(1+x^2) + 8cos(1.2(t-1)), v~N(0,5), r~N(0,16)
        return np.array([0.9, 10.0, 8.0, 1.2, -1.0, 5.0, 16.0, 0.05])
    return np.array([0.5, 25.0, 8.0, 1.2, 0.0, 10.0, 1.0, 0.05])


def make_ngm1d(B=1, T=50, N=32, L=50, step=0.05, seed=1, paper_constants=False,
               bw_value=1.0, prior=PRIOR_MIXTURE) -> Workload:
    p = ngm1d_params(paper_constants)
    a, b, c, om, toff, q, r, hc = p
    x0 = np.zeros((B, 1)); y = np.zeros((B, T, 1), np.float32); truth = np.zeros((B, T + 1, 1))
    for s in range(B):
        g = _rng(1, s)
        x = g.normal(0.0, np.sqrt(5.0))
        x0[s, 0] = x
        truth[s, 0, 0] = x
        for t in range(1, T + 1):
            x = a * x + b * x / (1 + x * x) + c * np.cos(om * (t + toff)) + g.normal(0, np.sqrt(q))
            truth[s, t, 0] = x
            y[s, t - 1, 0] = hc * x * x + g.normal(0, np.sqrt(r))
    return Workload("ngm1d", MODEL_NGM1D, p, 1, 1, N, L, step, BW_MEDIAN_ITER, bw_value, prior,
                    seed, x0, y, np.full(B, T, np.int32), np.full(B, N, np.int32), truth)


# ------------------------------------------------------------- range_cv ----
def range_params(beacons, dt=0.1, q=0.01, r=0.25) -> np.ndarray:
    beacons = np.asarray(beacons, np.float64)
    return np.concatenate([[dt, q, q, q, q, r, len(beacons)], beacons.ravel()])


def _cv_step(x, dt, g, q):
    f = np.array([x[0] + dt * x[2], x[1] + dt * x[3], x[2], x[3]])
    return f + g.normal(0.0, np.sqrt(q), 4)


def make_range_cv(B=1024, T=200, N=256, L=30, step=0.005, seed=2, dropout=(60, 120),
                  bw_value=1.0, prior=PRIOR_MIXTURE, first=0) -> Workload:
    beacons = _rng(2, 999_999).uniform(0.0, 100.0, (3, 2))
    p = range_params(beacons)
    dt, q, r = p[0], p[1], p[5]
    x0 = np.zeros((B, 4)); y = np.zeros((B, T, 3), np.float32); truth = np.zeros((B, T + 1, 4))
    for s in range(B):
        g = _rng(2, first + s)
        x = np.concatenate([g.uniform(25.0, 75.0, 2), g.normal(0.0, 1.0, 2)])
        x0[s] = x
        truth[s, 0] = x
        for t in range(1, T + 1):
            x = _cv_step(x, dt, g, q)
            truth[s, t] = x
            rho = np.hypot(x[0] - beacons[:, 0], x[1] - beacons[:, 1])
            z = rho + g.normal(0.0, np.sqrt(r), 3)
            if dropout is not None and dropout[0] <= t <= dropout[1]:
                z[1:] = np.nan
            y[s, t - 1] = z
    return Workload("range_cv", MODEL_RANGE_CV2D, p, 4, 3, N, L, step, BW_MEDIAN_ITER, bw_value,
                    prior, seed, x0, y, np.full(B, T, np.int32), np.full(B, N, np.int32), truth)


# ----------------------------------------------------------- clutter_cv ----
def clutter_params(dt=0.1, q=0.01, r=0.5, M=10, beta=0.2, area=100.0 * 100.0) -> np.ndarray:
    return np.array([dt, q, q, q, q, r, M, beta, area])


def make_clutter_cv(B=4096, Tmin=50, Tmax=400, N=512, L=30, step=0.005, seed=3, M=10,
                    p_miss=0.2, bw_value=1.0, prior=PRIOR_MIXTURE, uneven_N=None, first=0) -> Workload:
    p = clutter_params(M=M)
    dt, q, r = p[0], p[1], p[5]
    lengths = _rng(3, 888_888).integers(Tmin, Tmax + 1, B).astype(np.int32)
    maxT = int(lengths.max())
    x0 = np.zeros((B, 4)); y = np.full((B, maxT, 2 * M), np.nan, np.float32)
    truth = np.full((B, maxT + 1, 4), np.nan)
    for s in range(B):
        g = _rng(3, first + s)
        x = np.concatenate([g.uniform(-20.0, 20.0, 2), g.normal(0.0, 1.0, 2)])
        x0[s] = x
        truth[s, 0] = x
        for t in range(1, int(lengths[s]) + 1):
            x = _cv_step(x, dt, g, q)
            truth[s, t] = x
            pts = g.uniform(-50.0, 50.0, (M, 2))
            if g.uniform() >= p_miss:
                pts[g.integers(0, M)] = x[:2] + g.normal(0.0, np.sqrt(r), 2)
            y[s, t - 1] = pts.ravel()
    Nseq = np.full(B, N, np.int32)
    if uneven_N is not None:
        Nseq = _rng(3, 777_777).integers(uneven_N[0], uneven_N[1] + 1, B).astype(np.int32)
    return Workload("clutter_cv", MODEL_CLUTTER_CV2D, p, 4, 2 * M, int(Nseq.max()), L, step,
                    BW_MEDIAN_ITER, bw_value, prior, seed, x0, y, lengths, Nseq, truth)


# ----------------------------------------------------------- planar_arm ----
def arm_params(nl=7, dt=0.02, r=1e-4, qp=1.0, qv=0.01, link=0.3) -> np.ndarray:
    qa = qp * dt * dt
    return np.concatenate([[dt, nl, r], [qa] * nl, [qv] * nl, [link] * nl])


def _arm_fk(qang, lengths):
    th = np.cumsum(qang)
    return np.array([np.sum(lengths * np.cos(th)), np.sum(lengths * np.sin(th))])


def make_planar_arm(B=256, T=100, N=1024, L=50, step=1e-5, seed=4, nl=7, bw_value=1.0,
                    prior=PRIOR_MIXTURE, first=0) -> Workload:
    p = arm_params(nl=nl)
    dt, r = p[0], p[2]
    qv = p[3: 3 + 2 * nl]
    lengths = p[3 + 2 * nl:]
    d = 2 * nl
    x0 = np.zeros((B, d)); y = np.zeros((B, T, 2), np.float32); truth = np.zeros((B, T + 1, d))
    for s in range(B):
        g = _rng(4, first + s)
        x = np.concatenate([g.uniform(-0.5, 0.5, nl), np.zeros(nl)])
        x0[s] = x
        truth[s, 0] = x
        for t in range(1, T + 1):
            f = np.concatenate([x[:nl] + dt * x[nl:], x[nl:]])
            x = f + g.normal(0.0, 1.0, d) * np.sqrt(qv)
            truth[s, t] = x
            y[s, t - 1] = _arm_fk(x[:nl], lengths) + g.normal(0.0, np.sqrt(r), 2)
    return Workload("planar_arm", MODEL_PLANAR_ARM, p, d, 2, N, L, step, BW_MEDIAN_ITER, bw_value,
                    prior, seed, x0, y, np.full(B, T, np.int32), np.full(B, N, np.int32), truth)


# --------------------------------------------------------- linear_gauss ----
def linear_params(dt=0.1, q=0.01, r=0.05) -> np.ndarray:
    return np.array([dt, q, q, q, q, r])


def make_linear_gauss(B=1, T=20, N=64, L=100, step=0.002, seed=5, q=0.01, r=0.05,
                      bw_value=1.0, prior=PRIOR_MIXTURE) -> Workload:
    p = linear_params(q=q, r=r)
    dt = p[0]
    x0 = np.zeros((B, 4)); y = np.zeros((B, T, 2), np.float32); truth = np.zeros((B, T + 1, 4))
    for s in range(B):
        g = _rng(5, s)
        x = np.concatenate([g.uniform(-5.0, 5.0, 2), g.normal(0.0, 1.0, 2)])
        x0[s] = x
        truth[s, 0] = x
        for t in range(1, T + 1):
            x = _cv_step(x, dt, g, q)
            truth[s, t] = x
            y[s, t - 1] = x[:2] + g.normal(0.0, np.sqrt(r), 2)
    return Workload("linear_gauss", MODEL_LINEAR_GAUSS, p, 4, 2, N, L, step, BW_MEDIAN_ITER,
                    bw_value, prior, seed, x0, y, np.full(B, T, np.int32), np.full(B, N, np.int32),
                    truth)


FULL = {
    "ngm1d": lambda: make_ngm1d(),
    "range_cv": lambda: make_range_cv(),
    "clutter_cv": lambda: make_clutter_cv(),
    "planar_arm": lambda: make_planar_arm(),
}


# ------------------------------------------------------------- range_zv ----
ZV_ANCHORS = np.array([[5.0, 10.0], [0.0, 0.0], [10.0, 0.0]])
# (first step, length) of the periods in which anchor 1 is not heard; the
# lengths are Section V-C's blocking durations (2.5 .. 5 s at 10 Hz)
ZV_BLOCKED = ((50, 25), (150, 50), (250, 40), (350, 40), (450, 30), (530, 35))


def zv_params(anchors=ZV_ANCHORS, q=0.01, r=0.25) -> np.ndarray:
    anchors = np.asarray(anchors, np.float64)
    return np.concatenate([[q, q, r, len(anchors)], anchors.ravel()])


def make_range_zv(B=1, T=600, N=40, L=100, step=0.005, seed=6, blocked=ZV_BLOCKED, bw_value=1.0,
                  prior=PRIOR_MIXTURE, first=0) -> Workload:
    p = zv_params()
    q, r = p[0], p[2]
    anchors = p[4:].reshape(-1, 2)
    x0 = np.zeros((B, 2)); y = np.zeros((B, T, len(anchors)), np.float32); truth = np.zeros((B, T + 1, 2))
    for s in range(B):
        g = _rng(6, first + s)
        x = np.array([5.0, 4.0]) + g.normal(0.0, 0.5, 2)
        x0[s] = x
        truth[s, 0] = x
        for t in range(1, T + 1):
            x = x + g.normal(0.0, np.sqrt(q), 2)
            truth[s, t] = x
            y[s, t - 1] = np.linalg.norm(anchors - x, axis=1) + g.normal(0.0, np.sqrt(r), len(anchors))
        for t0, n in blocked or ():
            y[s, t0:min(T, t0 + n), 0] = np.nan
    return Workload("range_zv", MODEL_RANGE_ZV2D, p, 2, len(anchors), N, L, step, BW_MEDIAN_ITER, bw_value,
                    prior, seed, x0, y, np.full(B, T, np.int32), np.full(B, N, np.int32), truth)


# --------------------------------------------------------------- se2_rb ----
# Four landmarks around the 10 m reference circle (the paper shows four but
# gives no coordinates; these positions are chosen here).
SE2_LANDMARKS = np.array([[12.0, 12.0], [-12.0, 12.0], [-12.0, -12.0], [12.0, -12.0]])


def se2_params(landmarks=SE2_LANDMARKS, dt=0.1, alpha=(0.3, 0.3, 0.105), sr=1.0, sb=0.44, v=1.0,
               w=0.1) -> np.ndarray:
    """Section V-B: Q = diag((alpha dt)^2), range / bearing noise sr, sb."""
    landmarks = np.asarray(landmarks, np.float64)
    q = [(a * dt) ** 2 for a in alpha]
    return np.concatenate([[dt], q, [sr * sr, sb * sb, v, w, len(landmarks)], landmarks.ravel()])


def _wrap(a):
    return (a + np.pi) % (2.0 * np.pi) - np.pi


def make_se2_rb(B=10, T=630, N=20, L=100, step=1e-4, seed=7, outlier_p=0.1, outlier_scale=4.0,
                bw_value=1.0, prior=PRIOR_MIXTURE, first=0) -> Workload:
    """Truth: x_0 ~ N((10, 0, pi/2), diag(0.2^2, 0.2^2, 0.035^2)), then the
    noisy SE(2) motion; each step one landmark drawn uniformly, its range and
    bearing with N(0, sr^2) / N(0, sb^2) noise, each replaced by a draw with
    outlier_scale times the deviation with probability outlier_p.
    The default SVGD step is 1e-4, not the paper's 0.005: with Q = diag(0.03^2,
    0.03^2, 0.0105^2) the prior's curvature reaches 9070 in the heading and a
    plain SVGD step must stay below 2 / 9070 to contract."""
    p = se2_params()
    dt, q, sr, sb, v, w = p[0], p[1:4], np.sqrt(p[4]), np.sqrt(p[5]), p[6], p[7]
    lm = p[9:].reshape(-1, 2)
    x0 = np.zeros((B, 3)); y = np.zeros((B, T, 2), np.float32); truth = np.zeros((B, T + 1, 3))
    for s in range(B):
        g = _rng(7, first + s)
        x = np.array([10.0, 0.0, np.pi / 2]) + g.normal(0.0, 1.0, 3) * np.array([0.2, 0.2, 0.035])
        x0[s] = x
        truth[s, 0] = x
        for t in range(1, T + 1):
            th = x[2] + w * dt
            x = np.array([x[0] + v * dt * np.cos(th), x[1] + v * dt * np.sin(th), th]) + g.normal(0.0, np.sqrt(q))
            truth[s, t] = x
            l = g.integers(0, len(lm))
            nr = g.normal(0.0, sr) * (outlier_scale if g.random() < outlier_p else 1.0)
            nb = g.normal(0.0, sb) * (outlier_scale if g.random() < outlier_p else 1.0)
            dx, dy = x[0] - lm[l, 0], x[1] - lm[l, 1]
            y[s, t - 1] = [np.hypot(dx, dy) + nr, _wrap(np.arctan2(dy, dx) + nb)]
    return Workload("se2_rb", MODEL_SE2_RB, p, 3, 2, N, L, step, BW_MEDIAN_ITER, bw_value, prior, seed,
                    x0, y, np.full(B, T, np.int32), np.full(B, N, np.int32), truth)
