"""The exact median of the bandwidth rule (the median heuristic of Section V
and the Table Ex6 caption) on the GPU, path by path, against the oracle's
sort-based median: every search path of the kernel (the bracket around the
previous median, the 256-bin histogram locate, its refining second histogram,
the radix select) is driven by an input built for it, its counter must show
that it ran, and the bandwidth of every iteration must equal the oracle's
(relative 1e-5), as must the particles after the iterations."""
import numpy as np
import pytest

from paper_2312_08684_gb300 import Estimator, _binding as abi, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def rel_err(a, b):
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(1.0, np.sqrt(np.mean(b * b))))


def _run(oracle, wl, t, xprev, xinit, iters):
    """iters SVGD iterations at step t from xinit (GPU debug entry and
    oracle); returns the GPU's median-path counters."""
    m = oracle.Model(wl.kind, wl.params)
    y = np.ascontiguousarray(wl.y[:, t - 1])
    with Estimator.from_workload(wl) as est:
        xg, hg = est.debug_svgd(t, xprev, xinit, y, iters)
        counts = abi.smap_debug_median_stats(est.h)
    for b in range(wl.B):
        fprev = np.array([m.transition(t, v) for v in xprev[b].astype(np.float64)])
        xo, ho = m.svgd_iters(wl.prior, wl.bw_rule, wl.bw_value, t, y[b].astype(np.float64), fprev,
                              xinit[b].astype(np.float64), iters, wl.step)
        assert np.allclose(hg[b], ho, rtol=1e-5), (b, hg[b], ho)
        assert rel_err(xg[b], xo) <= 2e-5, (b, rel_err(xg[b], xo))
    return counts


def _range_sets(N, seed):
    wl = W.make_range_cv(B=2, T=6, N=N, L=1, dropout=None)
    rng = np.random.default_rng(seed)
    t = 3
    xprev = (wl.truth[:, t - 1, None, :] + 0.3 * rng.normal(0, 1, (wl.B, N, 4))).astype(np.float32)
    xinit = (wl.truth[:, t, None, :] + 0.3 * rng.normal(0, 1, (wl.B, N, 4))).astype(np.float32)
    return wl, t, xprev, xinit


def test_usual_sets_locate_then_bracket(oracle):
    """A fresh set: the histogram locates the middle ranks; later iterations
    find them in the bracket around the previous median."""
    wl, t, xprev, xinit = _range_sets(256, 1)
    c = _run(oracle, wl, t, xprev, xinit, 4)
    assert c[1] == wl.B and c[0] == 3 * wl.B and c[2] == 0


def test_duplicated_particles_take_the_radix_select(oracle):
    """Four distinct points, each held by 64 particles: 4096 pair distances tie
    at the median (more than the 2048 candidates a bracket keeps), and the
    copies stay identical under SVGD, so every iteration needs the radix
    select; the median is still exact."""
    wl, t, xprev, xinit = _range_sets(256, 2)
    for b in range(wl.B):
        xinit[b] = np.repeat(xinit[b, :4], 64, axis=0)
    c = _run(oracle, wl, t, xprev, xinit, 2)
    assert c[2] == 2 * wl.B and c[0] == 0


def test_far_outliers_defeat_the_guess(oracle):
    """The 32 particles that the first median guess pairs with others sit 10
    units (100 process-noise standard deviations) from the rest, each in its
    own direction (so every pair distance that involves one of them is far
    above the median): the guess (a mean of those pair distances) is more than
    4 octaves above the median, the histogram around it cannot locate the
    middle ranks, and the radix select takes over; the next iteration
    brackets the exact median.

    (Pair distances are formed as |x_i|^2 + |x_k|^2 - 2 x_i . x_k in FP32, so
    a tight cluster far from the centre of the set gets distances with an
    absolute error of a few u (|x_i|^2 + |x_k|^2); the outliers here are
    spread out, which keeps every distance near the median exact enough.)"""
    wl, t, xprev, xinit = _range_sets(256, 3)
    far = (7 * np.arange(32)) % 256
    ang = 2.0 * np.pi * np.arange(32) / 32.0
    xinit[:, far, 0] += (10.0 * np.cos(ang)).astype(np.float32)
    xinit[:, far, 1] += (10.0 * np.sin(ang)).astype(np.float32)
    c = _run(oracle, wl, t, xprev, xinit, 2)
    assert c[2] == wl.B and c[0] == wl.B


def test_many_keys_per_bin_take_the_refining_histogram(oracle):
    """N = 1024 particles of the 14-D arm state: 523,776 pair distances,
    concentrated enough that the located bins hold more than 2048 keys, so the
    second, refining histogram narrows them before the exact selection."""
    wl = W.make_planar_arm(B=2, T=6, N=1024, L=1)
    rng = np.random.default_rng(4)
    t = 3
    xprev = (wl.truth[:, t - 1, None, :] + 0.02 * rng.normal(0, 1, (wl.B, wl.N, wl.d))).astype(np.float32)
    xinit = (wl.truth[:, t, None, :] + 0.02 * rng.normal(0, 1, (wl.B, wl.N, wl.d))).astype(np.float32)
    c = _run(oracle, wl, t, xprev, xinit, 2)
    assert c[1] >= wl.B and c[3] >= wl.B and c[2] == 0
