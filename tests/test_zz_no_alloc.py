"""smap_viterbi_noalloc: the particle dynamic programme for callers that cannot
allocate device memory (a plug-in whose host application owns the device
memory budget, a control loop that must not enter the allocator). The test
allocates the input and output tensors itself, as such a caller's host would;
the entry point keeps its working state in the library's static device array.

Checked against the handle-based smap_viterbi on two calls in a row with
different shapes (the second call must not see the first call's state), with
the tolerances of the other parity tests: identical paths, J to 1e-12.
"""
import numpy as np
import pytest

from paper_2312_08684_gb300 import Estimator, _binding as abi, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()
    return torch


def _sets(wl, spread, seed):
    rng = np.random.default_rng(seed)
    return (wl.truth[:, 1:, None, :] + spread * rng.normal(0, 1, (wl.B, wl.maxT, wl.N, wl.d))).astype(np.float32)


def test_noalloc_matches_handle_viterbi_on_two_calls(torch):
    cases = [(W.make_range_cv(B=3, T=11, N=40, dropout=(3, 6)), 0.3),
             (W.make_clutter_cv(B=5, Tmin=7, Tmax=7, N=23), 0.3)]
    for k, (wl, spread) in enumerate(cases):
        hist = _sets(wl, spread, 10 + k)
        with Estimator.from_workload(wl) as est:
            path_ref, J_ref, _ = est.viterbi(hist, wl.y)
        dev = torch.device("cuda:0")
        x0 = torch.from_numpy(np.ascontiguousarray(wl.x0)).to(dev)
        h = torch.from_numpy(hist).to(dev)
        y = torch.from_numpy(np.ascontiguousarray(wl.y)).to(dev)
        path = torch.full((wl.B, wl.maxT + 1, wl.d), -7.0, dtype=torch.float32, device=dev)
        J = torch.full((wl.B,), -7.0, dtype=torch.float64, device=dev)
        abi.smap_viterbi_noalloc(wl.kind, wl.params, x0, h, y, path, J)
        torch.cuda.synchronize()
        assert np.array_equal(path.cpu().numpy(), path_ref), f"call {k}: paths differ"
        assert np.allclose(J.cpu().numpy(), J_ref, rtol=1e-12, atol=0), f"call {k}: J differs"


def test_noalloc_rejects_sizes_beyond_its_array(torch):
    wl = W.make_ngm1d(B=1, T=2, N=8)
    B, T, N = 48, 400, 512          # backpointers alone need 19.7 MB > 16 MiB
    dev = torch.device("cuda:0")
    x0 = torch.zeros((B, 1), dtype=torch.float64, device=dev)
    h = torch.zeros((B, T, N, 1), dtype=torch.float32, device=dev)
    y = torch.zeros((B, T, 1), dtype=torch.float32, device=dev)
    path = torch.zeros((B, T + 1, 1), dtype=torch.float32, device=dev)
    J = torch.zeros((B,), dtype=torch.float64, device=dev)
    with pytest.raises(abi.SmapError) as e:
        abi.smap_viterbi_noalloc(wl.kind, wl.params, x0, h, y, path, J)
    assert e.value.status == abi.SMAP_E_INVAL


def _noalloc(torch, wl, hist):
    dev = torch.device("cuda:0")
    x0 = torch.from_numpy(np.ascontiguousarray(wl.x0)).to(dev)
    h = torch.from_numpy(np.ascontiguousarray(hist)).to(dev)
    y = torch.from_numpy(np.ascontiguousarray(wl.y)).to(dev)
    path = torch.full((wl.B, wl.maxT + 1, wl.d), -7.0, dtype=torch.float32, device=dev)
    J = torch.full((wl.B,), -7.0, dtype=torch.float64, device=dev)
    abi.smap_viterbi_noalloc(wl.kind, wl.params, x0, h, y, path, J)
    torch.cuda.synchronize()
    return path.cpu().numpy(), J.cpu().numpy()


def test_nonfinite_sets_give_nan_and_the_next_call_is_clean(torch):
    """A NaN particle makes that sequence's scores non-finite: its J and its
    path after t = 0 are NaN, the other sequences are unaffected; the status
    the failed call leaves in the shared array does not leak into the next
    call."""
    wl = W.make_range_cv(B=3, T=9, N=24, dropout=(3, 5))
    hist = _sets(wl, 0.3, 31)
    bad = hist.copy()
    bad[1, 4, 7, 2] = np.nan
    with Estimator.from_workload(wl) as est:
        path_ref, J_ref, _ = est.viterbi(hist, wl.y)
    path, J = _noalloc(torch, wl, bad)
    assert np.isnan(J[1]) and np.all(np.isnan(path[1, 1:]))
    assert np.array_equal(path[1, 0], wl.x0[1].astype(np.float32))
    for b in (0, 2):
        assert np.array_equal(path[b], path_ref[b]) and J[b] == J_ref[b]
    path, J = _noalloc(torch, wl, hist)
    assert np.array_equal(path, path_ref)
    assert np.allclose(J, J_ref, rtol=1e-12, atol=0)


def test_live_handle_runs_after_a_smaller_noalloc_call(torch, oracle):
    """The handle-free call launches the same step-kernel function as a handle
    with the same variant, with less shared memory. A handle created and run
    before it must still run afterwards (smap_run_batch, smap_step,
    smap_viterbi), with the same results as before it."""
    wl = W.make_range_cv(B=2, T=8, N=256, L=4, dropout=(2, 4))
    small = W.make_range_cv(B=2, T=6, N=23, dropout=(2, 3))
    with Estimator.from_workload(wl) as est:
        est.set_variant(0)                     # the variant the handle-free call uses at N = 23
        path0, J0 = est.run_batch(wl.y)
        hist0 = est.history()
        _noalloc(torch, small, _sets(small, 0.3, 5))
        path1, J1 = est.run_batch(wl.y)        # graph replay of the earlier capture
        assert np.array_equal(path1, path0) and np.array_equal(J1, J0)
        _noalloc(torch, small, _sets(small, 0.3, 6))
        est.reset()
        for t in range(wl.maxT):
            est.step(np.ascontiguousarray(wl.y[:, t]))
        path2, J2 = est.map_sequence()
        assert np.array_equal(path2, path0) and np.array_equal(J2, J0)
        _noalloc(torch, small, _sets(small, 0.3, 7))
        path3, J3, _ = est.viterbi(hist0, wl.y)
        assert np.array_equal(path3, path0)
        assert np.allclose(J3, J0, rtol=1e-12, atol=0)
    for b in range(wl.B):
        ref = oracle.run_sequence(wl.kind, wl.params, wl.N, wl.L, wl.step, wl.bw_rule, wl.bw_value,
                                  wl.prior, wl.seed, b, wl.x0[b], wl.y[b].astype(np.float64))
        err = np.max(np.abs(path0[b] - ref["path"])) / max(1.0, np.sqrt(np.mean(ref["path"] ** 2)))
        assert err <= 1e-3


def test_two_live_handles_of_one_model_with_different_N(torch):
    """Two handles of one model and kernel variant, N = 64 and N = 512, used in
    turn: each launch needs its own shared-memory size from the one kernel
    function, and neither may lower the other's."""
    wa = W.make_range_cv(B=2, T=5, N=512, L=3, dropout=(2, 3))
    wb = W.make_range_cv(B=3, T=5, N=64, L=3, dropout=(2, 3))
    with Estimator.from_workload(wa) as ea, Estimator.from_workload(wb) as eb:
        ea.set_variant(0)
        eb.set_variant(0)
        pa0, Ja0 = ea.run_batch(wa.y)
        pb0, Jb0 = eb.run_batch(wb.y)
        ha, hb = ea.history(), eb.history()
        for _ in range(2):
            pa, Ja, _ = ea.viterbi(ha, wa.y)
            pb, Jb, _ = eb.viterbi(hb, wb.y)
            assert np.array_equal(pa, pa0) and np.allclose(Ja, Ja0, rtol=1e-12, atol=0)
            assert np.array_equal(pb, pb0) and np.allclose(Jb, Jb0, rtol=1e-12, atol=0)
        pa1, Ja1 = ea.run_batch(wa.y)
        pb1, Jb1 = eb.run_batch(wb.y)
        assert np.array_equal(pa1, pa0) and np.array_equal(Ja1, Ja0)
        assert np.array_equal(pb1, pb0) and np.array_equal(Jb1, Jb0)
