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
